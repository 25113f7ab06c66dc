// k_nc_back.cu -- backprojection of the non-circular SF-TR and DD footprint
// projectors and of SF-TT, and the entries for both directions (the
// footprint and the dispatch are in k_nc.cuh).
#include "k_nc.cuh"

namespace ctp {

// ------------------------------------------------------------ back (gather)
// Views staged per round: few enough that the sinogram rows a warp reads
// for them stay in L1 while the thread runs over its voxels.
constexpr int kNcViews = 16;

// Thread = voxel column (i, j) over ZT voxels; per round of views the thread
// runs over its voxels one at a time (the per-voxel body appears once in the
// code, which keeps the kernel within the instruction cache) with the
// voxel's sum carried in shared memory between rounds.
// RECON: the recon-mode (FBP) backprojection with the normalised footprint
// as the interpolation: weight rc_w / depth^2 over the footprint's area x
// height (SF-TR and DD).
template <typename TIn, int KIND, int NA, int NB, int ZT, bool RECON = false>
__global__ void __launch_bounds__(128, 8)
nc_back(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino, void *__restrict__ vol,
        int out_t, int tiles_x, int nzc) {
    __shared__ CtView sview[kNcViews];
    __shared__ float acc[ZT][128];
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool active = i < g.nx && j < g.ny;
    const int kbeg = kc * ZT;
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc[q][tid] = 0.f;
    const size_t vstride = (size_t)g.nv * g.nu;
    const TIn *ys = sino + (size_t)bt * g.nview * vstride;
    for (int v0 = 0; v0 < g.nview; v0 += kNcViews) {
        const int nvc = min(kNcViews, g.nview - v0);
        __syncthreads();
        {
            const float4 *s4 = reinterpret_cast<const float4 *>(views + v0);
            float4 *d4 = reinterpret_cast<float4 *>(sview);
            constexpr int W = sizeof(CtView) / sizeof(float4);
            for (int t = tid; t < nvc * W; t += 128) d4[t] = __ldg(s4 + t);
        }
        __syncthreads();
        if (!active) continue;
#pragma unroll 1
        for (int kk = 0; kk < ZT; ++kk) {
            const int k = kbeg + kk;
            if (k >= g.nz) break;
            float a = acc[kk][tid];
            for (int vv = 0; vv < nvc; ++vv) {
                const CtView &V = sview[vv];
                const TIn *yv = ys + (size_t)(v0 + vv) * vstride;
                NcFp<NA, NB> P;
                nc_fp<KIND, NA, NB>(V, g, i, j, k, P);
                float s = 0.f;
                if (P.a0 >= 0 && P.a0 + NA <= g.nu) {
                    // the whole window on the detector: one row pointer and
                    // predicated loads of the footprint's cells (no branches)
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        const int b = P.b0 + q;
                        if (P.Fv[q] != 0.f && b >= 0 && b < g.nv) {
                            const TIn *row = yv + (size_t)b * g.nu + P.a0;
                            float rs = P.Fu[0] * ld(row, 0);
#pragma unroll
                            for (int c = 1; c < NA; ++c)
                                rs = fmaf(P.Fu[c], c < P.n ? ld(row, (size_t)c) : 0.f, rs);
                            s = fmaf(P.Fv[q], rs, s);
                        }
                    }
                } else {
                    // cells off the detector get weight 0 and a clamped
                    // (in-bounds) address; cells past the footprint are not read
                    int ac[NA];
                    float wu[NA];
#pragma unroll
                    for (int c = 0; c < NA; ++c) {
                        const int ca = P.a0 + c;
                        const bool in = ca >= 0 && ca < g.nu;
                        ac[c] = in ? ca : 0;
                        wu[c] = in ? P.Fu[c] : 0.f;
                    }
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        const int b = P.b0 + q;
                        if (P.Fv[q] != 0.f && b >= 0 && b < g.nv) {
                            const TIn *row = yv + (size_t)b * g.nu;
                            float rs = wu[0] * ld(row, (size_t)ac[0]);
#pragma unroll
                            for (int c = 1; c < NA; ++c) {
                                if (c >= P.n) break;
                                rs = fmaf(wu[c], ld(row, (size_t)ac[c]), rs);
                            }
                            s = fmaf(P.Fv[q], rs, s);
                        }
                    }
                }
                a = fmaf(RECON ? V.rc_w / (P.cn * P.cn * P.size) : P.amp, s, a);
            }
            acc[kk][tid] = a;
        }
    }
    if (!active) return;
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc[kk][tid], out_t);
    }
}

namespace {
template <typename TIn, int KIND, int NA, int NB> struct NcBack {
    static cudaError_t go(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                          cudaStream_t st) {
        constexpr int ZT = 8;
        const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + ZT - 1) / ZT;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        nc_back<TIn, KIND, NA, NB, ZT><<<grd, blk, 0, st>>>(g, views, static_cast<const TIn *>(in), out, out_t,
                                                          tiles_x, nzc);
        return cudaGetLastError();
    }
};
}  // namespace

template <typename TIn, int KIND, int NA, int NB> struct NcBackRecon {
    static cudaError_t go(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                          cudaStream_t st) {
        constexpr int ZT = 8;
        const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + ZT - 1) / ZT;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        nc_back<TIn, KIND, NA, NB, ZT, true><<<grd, blk, 0, st>>>(g, views, static_cast<const TIn *>(in), out,
                                                                  out_t, tiles_x, nzc);
        return cudaGetLastError();
    }
};

cudaError_t launch_nc_recon(int dd, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                            void *out, int batch, cudaStream_t st) {
    const int kind = dd ? NC_DD : NC_SF;
    if (!nc_footprint_fits(g, kind)) return cudaErrorNotSupported;
    return nc_dispatch<NcBackRecon>(kind, in_t, g, views, in, out, out_t, batch, st);
}

cudaError_t launch_nc_back(int kind, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                           void *out, int batch, cudaStream_t st) {
    return nc_dispatch<NcBack>(kind, in_t, g, views, in, out, out_t, batch, st);
}

bool nc_footprint_fits(const CtGrid &g, int kind) {
    // at most 8 cells (half width <= 3.5) by 4 rows (half height <= 1.5)
    return (kind == NC_DD ? g.max_m_dd_u : g.max_m_sf_u) <= 3.5f &&
           (kind == NC_TT ? g.max_m_tt_v : g.max_m_sf_v) <= 1.5f;
}

cudaError_t launch_nc(int kind, int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st) {
    return dir == 0 ? launch_nc_fwd(kind, g, views, in_t, in, out_t, out, batch, st)
                    : launch_nc_back(kind, g, views, in_t, in, out_t, out, batch, st);
}

// SF-TT: the back direction scales the sinogram by each cell's amplitude into
// a stream-ordered FP32 workspace first.  Circular flat 3D geometry takes the
// column-walk kernels of k_sf.cu (the transaxial footprint is reused down
// each column), every other flat geometry the per-voxel footprint kernels.
template <typename TIn>
__global__ void __launch_bounds__(256)
tt_prescale(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ y, float *__restrict__ yp,
            int batch) {
    const size_t nview_cells = (size_t)g.nv * g.nu;
    const size_t total = nview_cells * g.nview * batch;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % g.nu);
        const int b = (int)((t / g.nu) % g.nv);
        const int v = (int)((t / nview_cells) % g.nview);
        yp[t] = tt_amp(views[v], g, a, b) * ld(y, t);
    }
}

cudaError_t launch_sftt(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                        void *out, int batch, cudaStream_t st) {
    const bool circ = sftt_circ_fits(g);
    if (dir == 0)
        return circ ? launch_sftt_circ(0, g, views, in_t, in, out_t, out, batch, st)
                    : launch_nc(NC_TT, 0, g, views, in_t, in, out_t, out, batch, st);
    const size_t n = (size_t)g.nview * g.nv * g.nu * batch;
    float *yp = nullptr;
    cudaError_t e = workspace_alloc((void **)&yp, n * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const size_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152u * 64u ? want : 152u * 64u);
    switch (in_t) {
    case 0: tt_prescale<float><<<blocks, 256, 0, st>>>(g, views, static_cast<const float *>(in), yp, batch); break;
    case 1: tt_prescale<__half><<<blocks, 256, 0, st>>>(g, views, static_cast<const __half *>(in), yp, batch); break;
    default:
        tt_prescale<__nv_bfloat16><<<blocks, 256, 0, st>>>(g, views, static_cast<const __nv_bfloat16 *>(in), yp,
                                                           batch);
        break;
    }
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = circ ? launch_sftt_circ(1, g, views, 0, yp, out_t, out, batch, st)
                 : launch_nc(NC_TT, 1, g, views, 0, yp, out_t, out, batch, st);
    const cudaError_t ef = workspace_free(yp, st);
    return e != cudaSuccess ? e : ef;
}

}  // namespace ctp
