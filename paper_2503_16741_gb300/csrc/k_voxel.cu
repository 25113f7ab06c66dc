// k_voxel.cu -- voxel-driven projector (Peters 1981, cited in Sec. 2.3).
// A voxel is a point at its centre; it is projected to the detector and
// shared between the 2 (2D) or 4 (3D) nearest cells with bilinear weights.
// The amplitude spreads the voxel's mass over the local ray density:
//   3D  A = dx dy dz r D^2 / (rho^3 du dv)      2D  A = dx dy r D / (rho^2 du)
// with r = |X - s|, rho = (X - s).n (flat) or the distance of X from the
// source axis (curved), D = source-detector distance (radius if curved).
// The back kernel is the classic voxel-driven backprojector; the forward
// kernels are its exact adjoint in gather form: the streaming forward of
// k_sf.cu in circular geometry, vx_fwd_nc below in non-circular geometry.
#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

// non-circular: per voxel
struct VxVox {
    float fu, fv, amp;
    float den;  // depth (X - s).n
};
__device__ __forceinline__ VxVox vx_vox_nc(const CtView &V, const CtGrid &g, int i, int j, int k) {
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, fmaf(V.au[2], fk, V.au[3])));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, fmaf(V.an[2], fk, V.an[3])));
    const float cv = fmaf(V.av[0], fi, fmaf(V.av[1], fj, fmaf(V.av[2], fk, V.av[3])));
    VxVox P;
    P.fu = fmaf(V.Ku, cu / cn, V.Cu);
    P.fv = fmaf(V.Kv, cv / cn, V.Cv);
    const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
    const float wz = fmaf(fk, g.dz, V.o[2]);
    P.amp = vx_amp(g, V, sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz))), cn);
    P.den = cn;
    return P;
}

// hat weight of cell c for fractional position f: 1 - t at floor(f), t at floor(f)+1
__device__ __forceinline__ float hat(float f, int c) {
    const float f0 = floorf(f);
    const int d = c - (int)f0;
    const float t = f - f0;
    return d == 0 ? 1.f - t : (d == 1 ? t : 0.f);
}

// ------------------------------------------------------------ back (gather)
template <typename TIn>
__device__ __forceinline__ float bilinear(const TIn *yv, const CtGrid &g, float fu, float fv) {
    const float a0f = floorf(fu), b0f = floorf(fv);
    const int a0 = (int)a0f, b0 = (int)b0f;
    const float ta = fu - a0f, tb = fv - b0f;
    float s = 0.f;
#pragma unroll
    for (int db = 0; db < 2; ++db) {
        const int b = b0 + db;
        if (b < 0 || b >= g.nv) continue;
        const float hb = db ? tb : 1.f - tb;
        const TIn *row = yv + (size_t)b * g.nu;
        float r = 0.f;
        if (a0 >= 0 && a0 < g.nu) r = (1.f - ta) * ld(row, (size_t)a0);
        if (a0 + 1 >= 0 && a0 + 1 < g.nu) r = fmaf(ta, ld(row, (size_t)(a0 + 1)), r);
        s = fmaf(hb, r, s);
    }
    return s;
}

// RECON: the recon-mode (FBP) backprojection of filtered projections (Sec.
// 2.3): the same bilinear interpolation with the depth weight in place of the
// voxel-driven amplitude, rc_w / depth^2 (flat: dbeta R D / ((X-s).n)^2;
// curved: dbeta / rho^2), constant down a column in circular geometry.
// Circular geometry: a column's two cells and their hat weights hold for all
// its voxels, so each detector row the chunk reaches is filtered once along u
// into a thread-private slice of shared memory, and each voxel blends its two
// rows (the same operations, in the same order, as the per-voxel bilinear);
// chunks whose rows do not fit the slice take the per-voxel form.
template <typename TIn, bool CURVED, int ZT, bool RECON = false>
__global__ void __launch_bounds__(128, 8)
vx_back_circ(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
             void *__restrict__ vol, int out_t, int tiles_x, int nzc) {
    constexpr int NR = ZT + 1;  // rows floor(fv) - B .. + 1 of the chunk's voxels, B the first voxel's row
    __shared__ float Rs[NR][128];
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int kbeg = kc * ZT;
    const int kend = min(kbeg + ZT, g.nz);
    float acc[ZT];
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc[q] = 0.f;
    const size_t vstride = (size_t)g.nv * g.nu;
    const TIn *ys = sino + (size_t)bt * g.nview * vstride;
    for (int v = 0; v < g.nview; ++v) {
        const CtView &V = views[v];
        const VxCol C = vx_col<CURVED>(V, g, i, j);
        if (C.fu <= -1.f || C.fu >= (float)g.nu) continue;
        const TIn *yv = ys + (size_t)v * vstride;
        const float wr = RECON ? V.rc_w / (C.den * C.den) : 0.f;
        // rows of the chunk: fv rises with k (sv > 0)
        const float Bf = floorf(fmaf(C.sv, (float)kbeg, C.fv0));
        const int B = (int)Bf;
        const int eL = (int)floorf(fmaf(C.sv, (float)(kend - 1), C.fv0)) - B + 1;
        if (C.sv > 0.f && eL < NR) {
            const float a0f = floorf(C.fu);
            const int a0 = (int)a0f;
            const float ta = C.fu - a0f;
            // cells and rows off the detector weigh zero; their loads read a
            // clamped in-range address, so the loads carry no branches
            const float w0 = (a0 >= 0 && a0 < g.nu) ? 1.f - ta : 0.f;
            const float w1 = (a0 + 1 >= 0 && a0 + 1 < g.nu) ? ta : 0.f;
            const int ac0 = min(max(a0, 0), g.nu - 1), ac1 = min(max(a0 + 1, 0), g.nu - 1);
#pragma unroll 4
            for (int e = 0; e <= eL; ++e) {
                const int b = B + e;
                const TIn *row = yv + (size_t)min(max(b, 0), g.nv - 1) * g.nu;
                const float r = fmaf(w1, ld(row, (size_t)ac1), w0 * ld(row, (size_t)ac0));
                Rs[e][tid] = (b >= 0 && b < g.nv) ? r : 0.f;
            }
            // voxels in pairs, in packed FP32x2 arithmetic (each lane rounds
            // as the scalar form would)
#pragma unroll
            for (int kk = 0; kk < ZT; kk += 2) {
                const int k = kbeg + kk;
                if (k + 1 < kend) {
                    const float2 fv = __ffma2_rn(make_float2(C.sv, C.sv), make_float2((float)k, (float)(k + 1)),
                                                 make_float2(C.fv0, C.fv0));
                    const float2 bf = make_float2(floorf(fv.x), floorf(fv.y));
                    const float2 tb = __fadd2_rn(fv, make_float2(-bf.x, -bf.y));
                    const int e0 = min(max((int)bf.x - B, 0), NR - 2), e1 = min(max((int)bf.y - B, 0), NR - 2);
                    const float2 sb = __ffma2_rn(tb, make_float2(Rs[e0 + 1][tid], Rs[e1 + 1][tid]),
                                                 __fmul2_rn(__fadd2_rn(make_float2(1.f, 1.f), make_float2(-tb.x, -tb.y)),
                                                            make_float2(Rs[e0][tid], Rs[e1][tid])));
                    float2 amp;
                    if (RECON) {
                        amp = make_float2(wr, wr);
                    } else {
                        const float2 wz = __ffma2_rn(make_float2((float)k, (float)(k + 1)), make_float2(g.dz, g.dz),
                                                     make_float2(V.o[2], V.o[2]));
                        const float2 t = __ffma2_rn(wz, wz, make_float2(C.rxy2, C.rxy2));
                        amp = __fmul2_rn(make_float2(C.amp1, C.amp1),
                                         __fmul2_rn(t, make_float2(rsqrtf(t.x), rsqrtf(t.y))));
                    }
                    const float2 a2 = __ffma2_rn(amp, sb, make_float2(acc[kk], acc[kk + 1]));
                    acc[kk] = a2.x;
                    acc[kk + 1] = a2.y;
                } else if (k < kend) {
                    const float fv = fmaf(C.sv, (float)k, C.fv0);
                    const float bf = floorf(fv);
                    const float tb = fv - bf;
                    const int e0 = min(max((int)bf - B, 0), NR - 2);
                    const float sb = fmaf(tb, Rs[e0 + 1][tid], (1.f - tb) * Rs[e0][tid]);
                    acc[kk] = fmaf(RECON ? wr : vx_amp_col(C, g, V, k), sb, acc[kk]);
                }
            }
            continue;
        }
#pragma unroll
        for (int kk = 0; kk < ZT; ++kk) {
            const int k = kbeg + kk;
            if (k >= g.nz) break;
            const float fv = fmaf(C.sv, (float)k, C.fv0);
            acc[kk] = fmaf(RECON ? wr : vx_amp_col(C, g, V, k), bilinear(yv, g, C.fu, fv), acc[kk]);
        }
    }
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc[kk], out_t);
    }
}

template <typename TIn, int ZT, bool RECON = false>
__global__ void __launch_bounds__(128)
vx_back_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
           void *__restrict__ vol, int out_t, int tiles_x, int nzc) {
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int kbeg = kc * ZT;
    float acc[ZT];
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc[q] = 0.f;
    const size_t vstride = (size_t)g.nv * g.nu;
    const TIn *ys = sino + (size_t)bt * g.nview * vstride;
    for (int v = 0; v < g.nview; ++v) {
        const CtView &V = views[v];
        const TIn *yv = ys + (size_t)v * vstride;
#pragma unroll
        for (int kk = 0; kk < ZT; ++kk) {
            const int k = kbeg + kk;
            if (k >= g.nz) break;
            const VxVox P = vx_vox_nc(V, g, i, j, k);
            acc[kk] = fmaf(RECON ? V.rc_w / (P.den * P.den) : P.amp, bilinear(yv, g, P.fu, P.fv), acc[kk]);
        }
    }
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc[kk], out_t);
    }
}

// ------------------------------------------------------------ forward (gather)
// Non-circular geometry: cell (a, b) receives the voxels whose centre
// projects within one cell of it (circular geometries take the streaming
// forward of k_sf.cu, which shares each column's u position down z).
template <typename TIn>
__global__ void __launch_bounds__(256)
vx_fwd_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
          void *__restrict__ sino, int out_t, int tiles_u) {
    int bx = blockIdx.x;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int v = bx % g.nview;
    const int bt = bx / g.nview;
    const int a = tu * 32 + threadIdx.x;
    const int b = blockIdx.y * 8 + threadIdx.y;
    if (a >= g.nu || b >= g.nv) return;
    const CtView &V = views[v];
    const int main_y = V.main_y;
    const SlabCoef sc = slab_coef(V, main_y);
    const float m = 1.0f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    float acc = 0.f;
    for (int s = 0; s < nslab; ++s) {
        int l0, l1, k0, k1;
        if (!search_flat(V, sc, s, a - m, a + m, b - m, b + m, nlat, g.nz, l0, l1, k0, k1)) continue;
        for (int l = l0; l <= l1; ++l) {
            const int i = main_y ? l : s, j = main_y ? s : l;
            for (int k = k0; k <= k1; ++k) {
                const VxVox P = vx_vox_nc(V, g, i, j, k);
                const float w = hat(P.fu, a) * hat(P.fv, b);
                if (w == 0.f) continue;
                acc = fmaf(P.amp * w, ld(x, ((size_t)k * g.ny + j) * g.nx + i), acc);
            }
        }
    }
    st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc, out_t);
}

// ------------------------------------------------------------ launchers
namespace {
constexpr int kZT = 8;    // voxels per thread, non-circular back
constexpr int kZTc = 16;  // circular back

template <typename TIn>
cudaError_t vx_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                        int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (dir == 0) {
        const int tiles_u = (g.nu + 31) / 32;
        dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
        vx_fwd_nc<TIn><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
    } else {
        const int tiles_x = (g.nx + 31) / 32;
        const int nzc = (g.nz + kZT - 1) / kZT, nzcc = (g.nz + kZTc - 1) / kZTc;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        dim3 grdc((unsigned)(tiles_x * nzcc * batch), (unsigned)((g.ny + 3) / 4));
        if (g.variant == GEO_NONCIRC_FLAT)
            vx_back_nc<TIn, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
        else if (g.variant == GEO_CIRC_CURVED)
            vx_back_circ<TIn, true, kZTc><<<grdc, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzcc);
        else
            vx_back_circ<TIn, false, kZTc><<<grdc, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzcc);
    }
    return cudaGetLastError();
}
}  // namespace

namespace {
template <typename TIn>
cudaError_t vx_recon_t(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                       cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    const int tiles_x = (g.nx + 31) / 32;
    const int nzc = (g.nz + kZT - 1) / kZT, nzcc = (g.nz + kZTc - 1) / kZTc;
    dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
    dim3 grdc((unsigned)(tiles_x * nzcc * batch), (unsigned)((g.ny + 3) / 4));
    if (g.variant == GEO_NONCIRC_FLAT)
        vx_back_nc<TIn, kZT, true><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
    else if (g.variant == GEO_CIRC_CURVED)
        vx_back_circ<TIn, true, kZTc, true><<<grdc, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzcc);
    else
        vx_back_circ<TIn, false, kZTc, true><<<grdc, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzcc);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_voxel_recon(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return vx_recon_t<float>(g, views, in, out, out_t, batch, st);
    case 1: return vx_recon_t<__half>(g, views, in, out, out_t, batch, st);
    default: return vx_recon_t<__nv_bfloat16>(g, views, in, out, out_t, batch, st);
    }
}

cudaError_t launch_voxel(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                         int out_t, void *out, int batch, cudaStream_t st) {
    if (dir == 0 && g.variant != GEO_NONCIRC_FLAT)
        return launch_vx_fwd_circ(g, views, in_t, in, out_t, out, batch, st);
    switch (in_t) {
    case 0: return vx_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return vx_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return vx_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
