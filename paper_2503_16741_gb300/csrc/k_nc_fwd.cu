// k_nc_fwd.cu -- forward projection of the non-circular SF-TR and DD
// footprint projectors and of SF-TT (the footprint and the dispatch are in
// k_nc.cuh).
#include "k_nc.cuh"

namespace ctp {

// ------------------------------------------------------------ forward (gather)
// Index box of slab s for a detector window [Flo, Fhi] x [Glo, Ghi]: the
// window's four corner rays meet the slab plane at points whose lateral and
// axial indices are affine in s (the plane equations are affine in s and
// their 2 x 2 determinant does not depend on s), so the box of every slab
// comes from 8 coefficient pairs formed once per thread.
struct NcBox {
    float l0[4], l1[4], k0[4], k1[4];  // l = l0 + l1 s, k = k0 + k1 s per corner ray
};

__device__ __forceinline__ NcBox nc_box_coef(const CtView &V, const SlabCoef &c, float Flo, float Fhi,
                                             float Glo, float Ghi) {
    NcBox B;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float tu = (q ? Fhi : Flo) - V.Cu;
        const float Pl = fmaf(V.Ku, c.ul, -tu * c.nl);
        const float Pk = fmaf(V.Ku, c.uk, -tu * c.nk);
        const float P0 = fmaf(V.Ku, c.u3, -tu * c.n3), P1 = fmaf(V.Ku, c.us, -tu * c.ns);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float tv = (r ? Ghi : Glo) - V.Cv;
            const float Ql = fmaf(V.Kv, c.vl, -tv * c.nl);
            const float Qk = fmaf(V.Kv, c.vk, -tv * c.nk);
            const float Q0 = fmaf(V.Kv, c.v3, -tv * c.n3), Q1 = fmaf(V.Kv, c.vs, -tv * c.ns);
            const float rdet = 1.f / fmaf(Pl, Qk, -Pk * Ql);
            const int t = 2 * q + r;
            B.l0[t] = fmaf(-P0, Qk, Q0 * Pk) * rdet;
            B.l1[t] = fmaf(-P1, Qk, Q1 * Pk) * rdet;
            B.k0[t] = fmaf(-Q0, Pl, P0 * Ql) * rdet;
            B.k1[t] = fmaf(-Q1, Pl, P1 * Ql) * rdet;
        }
    }
    return B;
}

__device__ __forceinline__ bool nc_box(const NcBox &B, float s, int nlat, int nk, int &l0, int &l1, int &k0,
                                       int &k1) {
    float lmin = 3.0e38f, lmax = -3.0e38f, kmin = 3.0e38f, kmax = -3.0e38f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float l = fmaf(B.l1[t], s, B.l0[t]), k = fmaf(B.k1[t], s, B.k0[t]);
        lmin = fminf(lmin, l); lmax = fmaxf(lmax, l);
        kmin = fminf(kmin, k); kmax = fmaxf(kmax, k);
    }
    if (!(isfinite(lmin) && isfinite(lmax) && isfinite(kmin) && isfinite(kmax))) return false;
    l0 = max(0, (int)ceilf(lmin));
    l1 = min(nlat - 1, (int)floorf(lmax));
    k0 = max(0, (int)ceilf(kmin));
    k1 = min(nk - 1, (int)floorf(kmax));
    return l0 <= l1 && k0 <= k1;
}

// Footprint cache of one round: per voxel its NA transaxial weights times
// amplitude times value, its axial weights placed in an 8-row window that
// starts at a 4-row group boundary of the tile, and (first cell, group).
// Lateral index at which a line of constant fu meets row k of slab s:
// l = c0 + ck k + cs s (the line Ku (au.X) = (F - Cu) (an.X) in the slab plane).
struct NcLine {
    float c0, ck, cs;
};
__device__ __forceinline__ NcLine nc_line(const CtView &V, const SlabCoef &c, float F) {
    const float tu = F - V.Cu;
    const float rPl = -1.f / fmaf(V.Ku, c.ul, -tu * c.nl);
    return NcLine{fmaf(V.Ku, c.u3, -tu * c.n3) * rPl, fmaf(V.Ku, c.uk, -tu * c.nk) * rPl,
                  fmaf(V.Ku, c.us, -tu * c.ns) * rPl};
}

constexpr int kNcMaxV = 1024;  // voxels cached per round
constexpr int kNcViewBlock = 32;  // views of one tile adjacent in the grid

template <int NA> struct NcCache {
    float4 Fv[2][kNcMaxV];  // rows 4 g0 .. 4 g0 + 7 of the tile
    float Fu[NA][kNcMaxV];
    int2 ag[kNcMaxV];       // (a0, g0)
};

// Forward: CTA = 64 cells x 64 rows of one view, 256 threads; thread (tx, ty)
// owns cells A0 + 4 tx .. + 3 and rows B0 + 4 ty .. + 3 (16 sums).
template <typename TIn, int KIND, int NA, int NB>
__global__ void __launch_bounds__(256, 3)
nc_fwd(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol, const TIn *__restrict__ volZ,
       void *__restrict__ sino, int out_t, int tiles_u, int tiles_v) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    NcCache<NA> &S = *reinterpret_cast<NcCache<NA> *>(smem_raw);
    __shared__ NcBox tile;  // the CTA's box coefficients (read as broadcasts)
    // CTA order: kNcViewBlock consecutive views of one tile, then tiles, then
    // view blocks.  Neighbouring views of a tile read nearly the same voxels,
    // so CTAs resident together share their slabs in L2.
    int bx = blockIdx.x;
    const int vl = bx % kNcViewBlock; bx /= kNcViewBlock;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int tv = bx % tiles_v; bx /= tiles_v;
    const int nvb = (g.nview + kNcViewBlock - 1) / kNcViewBlock;
    const int v = (bx % nvb) * kNcViewBlock + vl;
    const int bt = bx / nvb;
    if (v >= g.nview) return;  // the last block's missing views (whole CTA)
    const int tid = threadIdx.y * 16 + threadIdx.x;
    const int A0 = tu * 64, B0 = tv * 64;
    const int a = A0 + 4 * threadIdx.x, ty = threadIdx.y, rb = B0 + 4 * ty;
    const CtView &V = views[v];
    const int main_y = V.main_y;
    const SlabCoef sc = slab_coef(V, main_y);
    const float mu = (KIND == NC_DD ? V.m_dd_u : V.m_sf_u) + 0.5f + kSearchPad;
    const float mv = (KIND == NC_TT ? V.m_tt_v : V.m_sf_v) + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const size_t nvox = (size_t)g.nx * g.ny * g.nz;
    const TIn *x = vol + (size_t)bt * nvox;
    const TIn *xz = volZ ? volZ + (size_t)bt * nvox : nullptr;
    if (tid == 0) tile = nc_box_coef(V, sc, A0 - mu, A0 + 63.f + mu, B0 - mv, B0 + 63.f + mv);
    const NcBox cell = nc_box_coef(V, sc, a - mu, a + 3.f + mu, rb - mv, rb + 3.f + mv);
    // the thread's u window per row k: between two lines of constant fu
    const NcLine ln1 = nc_line(V, sc, a - mu), ln2 = nc_line(V, sc, a + 3.f + mu);
    const bool lines = isfinite(ln1.c0) && isfinite(ln1.ck) && isfinite(ln1.cs) && isfinite(ln2.c0) &&
                       isfinite(ln2.ck) && isfinite(ln2.cs);
    const bool live = a < g.nu && rb < g.nv;
    // sums of rows rb + r, cells (a, a + 1) and (a + 2, a + 3): packed FP32x2
    float2 acc[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[r][c] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int s = 0; s < nslab; ++s) {
        const float fs = (float)s;
        int L0, L1, K0, K1;
        if (!nc_box(tile, fs, nlat, g.nz, L0, L1, K0, K1)) continue;  // uniform over the CTA
        int l0 = 0, l1 = -1, k0 = 0, k1 = -1;
        const bool mine = live && nc_box(cell, fs, nlat, g.nz, l0, l1, k0, k1);
        // rounds of nl x nk voxels, k fastest (contiguous in the z-major copy)
        const int nk = min(K1 - K0 + 1, kNcMaxV);
        const int nlr = kNcMaxV / nk;
        for (int kc = K0; kc <= K1; kc += nk) {
            const int nkr = min(nk, K1 - kc + 1);
            for (int lc = L0; lc <= L1; lc += nlr) {
                const int nl = min(nlr, L1 - lc + 1);
                __syncthreads();
                for (int idx = tid; idx < nl * nkr; idx += 256) {
                    const int l = lc + idx / nkr, k = kc + idx % nkr;
                    const int i = main_y ? l : s, j = main_y ? s : l;
                    NcFp<NA, NB> P;
                    nc_fp<KIND, NA, NB>(V, g, i, j, k, P);
                    const float xv = xz ? ld(xz, ((size_t)j * g.nx + i) * g.nz + k)
                                        : ld(x, ((size_t)k * g.ny + j) * g.nx + i);
                    const float w = P.amp * xv;
#pragma unroll
                    for (int q = 0; q < NA; ++q) S.Fu[q][idx] = P.Fu[q] * w;
                    // first 4-row group of the footprint and its offset in it
                    const int rel = P.b0 - B0;
                    const int g0 = rel >= 0 ? rel >> 2 : -((3 - rel) >> 2);
                    const int o = rel - 4 * g0;  // 0 .. 3
                    float w8[8];
#pragma unroll
                    for (int t = 0; t < 8; ++t) w8[t] = 0.f;
#pragma unroll
                    for (int oo = 0; oo < 4; ++oo)
                        if (o == oo) {
#pragma unroll
                            for (int q = 0; q < NB; ++q) w8[oo + q] = P.Fv[q];
                        }
                    S.Fv[0][idx] = make_float4(w8[0], w8[1], w8[2], w8[3]);
                    S.Fv[1][idx] = make_float4(w8[4], w8[5], w8[6], w8[7]);
                    S.ag[idx] = make_int2(P.a0, g0);
                }
                __syncthreads();
                if (!mine) continue;
                const int la = max(l0, lc), lb = min(l1, lc + nl - 1);
                const int ka = max(k0, kc), kb = min(k1, kc + nkr - 1);
                const float ls1 = fmaf(ln1.cs, fs, ln1.c0), ls2 = fmaf(ln2.cs, fs, ln2.c0);
                for (int k = ka; k <= kb; ++k) {
                    int lo = la, hi = lb;
                    if (lines) {  // lateral range of row k (1e-3 voxel rounding guard)
                        const float fk = (float)k;
                        const float u1 = fmaf(ln1.ck, fk, ls1), u2 = fmaf(ln2.ck, fk, ls2);
                        lo = max(la, (int)ceilf(fminf(u1, u2) - 1e-3f));
                        hi = min(lb, (int)floorf(fmaxf(u1, u2) + 1e-3f));
                    }
                    int idx = (lo - lc) * nkr + (k - kc);
                    for (int l = lo; l <= hi; ++l, idx += nkr) {
                        const int2 ag = S.ag[idx];
                        const int d = a - ag.x;  // first cell of the thread in the footprint
                        const int gd = ty - ag.y;
                        if ((unsigned)gd > 1u || (unsigned)(d + 3) >= (unsigned)(NA + 3)) continue;  // -4 < d < NA
                        const float4 fv = S.Fv[gd][idx];
                        // Fu[d + c][idx] for the thread's cells c: one base offset
                        const float *fu = &S.Fu[0][0];
                        const int off = d * kNcMaxV + idx;
                        float wu[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            wu[c] = (unsigned)(d + c) < (unsigned)NA ? fu[off + c * kNcMaxV] : 0.f;
                        const float2 w01 = make_float2(wu[0], wu[1]), w23 = make_float2(wu[2], wu[3]);
                        const float fr[4] = {fv.x, fv.y, fv.z, fv.w};
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float2 f = make_float2(fr[r], fr[r]);
                            acc[r][0] = __ffma2_rn(w01, f, acc[r][0]);
                            acc[r][1] = __ffma2_rn(w23, f, acc[r][1]);
                        }
                    }
                }
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int b = rb + r;
        if (b >= g.nv) break;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int ac = a + c;
            const float2 p = acc[r][c >> 1];
            const float sum = (c & 1) ? p.y : p.x;
            if (ac < g.nu)
                st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + ac,
                       KIND != NC_SF ? sum * nc_cell_factor<KIND>(V, g, ac, b) : sum, out_t);
        }
    }
}

namespace {
template <typename TIn, int KIND, int NA, int NB> struct NcFwd {
    static cudaError_t go(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                          cudaStream_t st) {
        const TIn *src = static_cast<const TIn *>(in);
        const size_t smem = sizeof(NcCache<NA>);
        cudaError_t e = cudaFuncSetAttribute(nc_fwd<TIn, KIND, NA, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        // a z-major copy of the volume (pooled workspace) makes each round's
        // reads contiguous along k; without it the reads are strided
        TIn *xZ = nullptr;
        const size_t n = (size_t)g.nx * g.ny * g.nz * batch;
        if (workspace_alloc((void **)&xZ, n * sizeof(TIn), st) != cudaSuccess) {
            cudaGetLastError();
            xZ = nullptr;
        } else if ((e = zmajor_copy(sizeof(TIn), src, xZ, g.nx, g.ny, g.nz, batch, st)) != cudaSuccess) {
            workspace_free(xZ, st);
            return e;
        }
        const int tiles_u = (g.nu + 63) / 64, tiles_v = (g.nv + 63) / 64;
        const size_t nvb = (g.nview + kNcViewBlock - 1) / kNcViewBlock;
        dim3 blk(16, 16), grd((unsigned)((size_t)kNcViewBlock * tiles_u * tiles_v * nvb * batch));
        nc_fwd<TIn, KIND, NA, NB><<<grd, blk, smem, st>>>(g, views, src, xZ, out, out_t, tiles_u, tiles_v);
        e = cudaGetLastError();
        if (xZ) {
            const cudaError_t ef = workspace_free(xZ, st);
            if (e == cudaSuccess) e = ef;
        }
        return e;
    }
};
}  // namespace

cudaError_t launch_nc_fwd(int kind, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                          void *out, int batch, cudaStream_t st) {
    return nc_dispatch<NcFwd>(kind, in_t, g, views, in, out, out_t, batch, st);
}

}  // namespace ctp
