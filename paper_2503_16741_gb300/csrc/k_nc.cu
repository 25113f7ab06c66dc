// k_nc.cu -- SF-TR and DD footprint projectors in non-circular geometry
// (flat detector with per-view tilt and in-plane rotation, Sec. 2.2), where a
// voxel's transaxial footprint changes with its z (the footprint methods cited
// in Sec. 2.3: Long, Fessler & Balter 2010; De Man & Basu 2004).  Every voxel
// carries its own footprint of at most NA cells by NB rows (NA = 4, 6 or 8,
// NB = 3 or 4, chosen by the launcher from the per-view footprint bounds;
// wider footprints go to the general kernels).
//   back:    thread = voxel column over a z-chunk, all views (records staged
//            in shared memory); per voxel and view the footprint, then its
//            NA x NB taps.
//   forward: CTA = 16 cells x 64 rows of one view.  Per slab of the view's
//            main axis the CTA computes, once, the footprint of every voxel
//            that can reach its tile into shared memory (a footprint cache);
//            each thread then gathers, for its cell and 4 rows, the cached
//            weights of the voxels in its own search box.
// Both are gathers with a fixed summation order: deterministic, no atomics.
// DD multiplies by the cell's path length after the forward gather; its back
// direction takes a sinogram already scaled by it.
#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

template <int NA, int NB> struct NcFp {
    int a0, b0;    // first cell, first row of the footprint
    float Fu[NA];  // transaxial weights of cells a0 .. a0 + NA - 1
    float Fv[NB];  // axial weights of rows b0 .. b0 + NB - 1
    float amp;     // SF amplitude dx |w| / max(|w_x|, |w_y|); DD: 1
};

// Footprint of voxel (i, j, k) in view V.  The centre is projected with a
// correctly rounded reciprocal; corner and end-point offsets are formed from
// small differences, Ku (du - r dn) / (cn + dn) with r = cu / cn, where a fast
// division's few ulp are ~1e-7 cell.
template <bool DD, int NA, int NB>
__device__ __forceinline__ void nc_fp(const CtView &V, const CtGrid &g, int i, int j, int k, NcFp<NA, NB> &P) {
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, fmaf(V.au[2], fk, V.au[3])));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, fmaf(V.an[2], fk, V.an[3])));
    const float cv = fmaf(V.av[0], fi, fmaf(V.av[1], fj, fmaf(V.av[2], fk, V.av[3])));
    const float rcn = __frcp_rn(cn);
    const float r = cu * rcn, rv = cv * rcn;
    int aref, bref;
    float fr, vr;
    split_cell(fmaf(V.Ku, r, V.Cu), aref, fr);
    split_cell(fmaf(V.Kv, rv, V.Cv), bref, vr);
    Trap T;
    if (DD) {  // boundary points +- half a voxel along the lateral axis
        const int q = V.main_y ? 0 : 1;
        const float hu = 0.5f * V.au[q], hn = 0.5f * V.an[q];
        const float e1 = fr + V.Ku * __fdividef(fmaf(r, hn, -hu), cn - hn);
        const float e2 = fr + V.Ku * __fdividef(fmaf(-r, hn, hu), cn + hn);
        const float lo = fminf(e1, e2), hi = fmaxf(e1, e2);
        T = make_trap(lo, lo, hi, hi);
    } else {  // the four transaxial corners, sorted into a trapezoid
        const float hxu = 0.5f * V.au[0], hxn = 0.5f * V.an[0];
        const float hyu = 0.5f * V.au[1], hyn = 0.5f * V.an[1];
        float t0 = fr + V.Ku * __fdividef(fmaf(-r, -hxn - hyn, -hxu - hyu), cn - hxn - hyn);
        float t1 = fr + V.Ku * __fdividef(fmaf(-r, hxn - hyn, hxu - hyu), cn + hxn - hyn);
        float t2 = fr + V.Ku * __fdividef(fmaf(-r, hyn - hxn, hyu - hxu), cn - hxn + hyn);
        float t3 = fr + V.Ku * __fdividef(fmaf(-r, hxn + hyn, hxu + hyu), cn + hxn + hyn);
        sort4(t0, t1, t2, t3);
        T = make_trap(t0, t1, t2, t3);
    }
    const int d0 = (int)floorf(T.k0 + 0.5f), d1 = (int)floorf(T.k3 + 0.5f);
    trap_cellsN<NA>(T, d0, d1, P.Fu);
    P.a0 = aref + d0;
    // axial rectangle: the end points (z -+ dz/2) at the voxel's (x, y) centre
    const float hzv = 0.5f * V.av[2], hzn = 0.5f * V.an[2];
    const float f1 = vr + V.Kv * __fdividef(fmaf(-rv, hzn, hzv), cn + hzn);
    const float f2 = vr + V.Kv * __fdividef(fmaf(rv, hzn, -hzv), cn - hzn);
    const float vlo = fminf(f1, f2), vhi = fmaxf(f1, f2);
    const int e0 = (int)floorf(vlo + 0.5f);
#pragma unroll
    for (int q = 0; q < NB; ++q) {
        const float e = (float)(e0 + q);
        P.Fv[q] = overlap(vlo, vhi, e - 0.5f, e + 0.5f);
    }
    P.b0 = bref + e0;
    if (DD) {
        P.amp = 1.f;
    } else {
        const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
        const float wz = fmaf(fk, g.dz, V.o[2]);
        const float t = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        P.amp = __fdividef(g.dx * t * rsqrtf(t), fmaxf(fabsf(wx), fabsf(wy)));
    }
}

// ------------------------------------------------------------ back (gather)
constexpr int kNcViews = 64;

template <typename TIn, bool DD, int NA, int NB, int ZT>
__global__ void __launch_bounds__(128, 6)
nc_back(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino, void *__restrict__ vol,
        int out_t, int tiles_x, int nzc) {
    __shared__ CtView sview[kNcViews];
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool active = i < g.nx && j < g.ny;
    const int kbeg = kc * ZT;
    float acc[ZT];
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc[q] = 0.f;
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
        for (int vv = 0; vv < nvc; ++vv) {
            const CtView &V = sview[vv];
            const TIn *yv = ys + (size_t)(v0 + vv) * vstride;
#pragma unroll
            for (int kk = 0; kk < ZT; ++kk) {
                const int k = kbeg + kk;
                if (k < g.nz) {
                    NcFp<NA, NB> P;
                    nc_fp<DD, NA, NB>(V, g, i, j, k, P);
                    // cells and rows off the detector get weight 0 and a clamped
                    // (in-bounds) address
                    int ac[NA];
                    float wu[NA];
#pragma unroll
                    for (int c = 0; c < NA; ++c) {
                        const int a = P.a0 + c;
                        const bool in = a >= 0 && a < g.nu;
                        ac[c] = in ? a : 0;
                        wu[c] = in ? P.Fu[c] : 0.f;
                    }
                    float s = 0.f;
#pragma unroll
                    for (int q = 0; q < NB; ++q) {
                        const int b = P.b0 + q;
                        if (P.Fv[q] != 0.f && b >= 0 && b < g.nv) {
                            const TIn *row = yv + (size_t)b * g.nu;
                            float rs = wu[0] * ld(row, (size_t)ac[0]);
#pragma unroll
                            for (int c = 1; c < NA; ++c) rs = fmaf(wu[c], ld(row, (size_t)ac[c]), rs);
                            s = fmaf(P.Fv[q], rs, s);
                        }
                    }
                    acc[kk] = fmaf(P.amp, s, acc[kk]);
                }
            }
        }
    }
    if (!active) return;
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc[kk], out_t);
    }
}

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

// voxels cached per round (the cache stays within 48 KB of static shared memory)
template <int NA, int NB> struct NcCache {
    static constexpr int MAXV = (NA + NB + 2) * 1024 * 4 < 48 * 1024 ? 1024 : 768;
    float Fu[NA][MAXV];   // transaxial weights x amplitude x voxel value
    float Fv[NB][MAXV];   // axial weights
    int a0[MAXV], b0[MAXV];
};

template <typename TIn, bool DD, int NA, int NB>
__global__ void __launch_bounds__(256, 3)
nc_fwd(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol, void *__restrict__ sino,
       int out_t, int tiles_u, int tiles_v) {
    __shared__ NcCache<NA, NB> S;
    constexpr int kNcMaxV = NcCache<NA, NB>::MAXV;
    __shared__ NcBox tile;  // the CTA's box coefficients (read as broadcasts)
    int bx = blockIdx.x;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int tv = bx % tiles_v; bx /= tiles_v;
    const int v = bx % g.nview;
    const int bt = bx / g.nview;
    const int tid = threadIdx.y * 16 + threadIdx.x;
    const int A0 = tu * 16, B0 = tv * 64;
    const int a = A0 + threadIdx.x, rb = B0 + 4 * threadIdx.y;
    const CtView &V = views[v];
    const int main_y = V.main_y;
    const SlabCoef sc = slab_coef(V, main_y);
    const float mu = (DD ? V.m_dd_u : V.m_sf_u) + 0.5f + kSearchPad, mv = V.m_sf_v + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    if (tid == 0) tile = nc_box_coef(V, sc, A0 - mu, A0 + 15.f + mu, B0 - mv, B0 + 63.f + mv);
    const NcBox cell = nc_box_coef(V, sc, a - mu, a + mu, rb - mv, rb + 3.f + mv);
    const bool live = a < g.nu && rb < g.nv;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    __syncthreads();
    for (int s = 0; s < nslab; ++s) {
        const float fs = (float)s;
        int L0, L1, K0, K1;
        if (!nc_box(tile, fs, nlat, g.nz, L0, L1, K0, K1)) continue;  // uniform over the CTA
        int l0 = 0, l1 = -1, k0 = 0, k1 = -1;
        const bool mine = live && nc_box(cell, fs, nlat, g.nz, l0, l1, k0, k1);
        for (int lc = L0; lc <= L1; lc += kNcMaxV) {
            const int nl = min(L1 - lc + 1, kNcMaxV);
            const int nkc = kNcMaxV / nl;
            for (int kc = K0; kc <= K1; kc += nkc) {
                const int nk = min(K1 - kc + 1, nkc);
                __syncthreads();
                for (int idx = tid; idx < nl * nk; idx += 256) {
                    const int l = lc + idx % nl, k = kc + idx / nl;
                    const int i = main_y ? l : s, j = main_y ? s : l;
                    NcFp<NA, NB> P;
                    nc_fp<DD, NA, NB>(V, g, i, j, k, P);
                    const float w = P.amp * ld(x, ((size_t)k * g.ny + j) * g.nx + i);
#pragma unroll
                    for (int q = 0; q < NA; ++q) S.Fu[q][idx] = P.Fu[q] * w;
#pragma unroll
                    for (int q = 0; q < NB; ++q) S.Fv[q][idx] = P.Fv[q];
                    S.a0[idx] = P.a0;
                    S.b0[idx] = P.b0;
                }
                __syncthreads();
                if (!mine) continue;
                const int la = max(l0, lc), lb = min(l1, lc + nl - 1);
                const int ka = max(k0, kc), kb = min(k1, kc + nk - 1);
                for (int k = ka; k <= kb; ++k) {
                    const int row = (k - kc) * nl - lc;
                    for (int l = la; l <= lb; ++l) {
                        const int idx = row + l;
                        const int d = a - S.a0[idx];
                        if ((unsigned)d >= (unsigned)NA) continue;
                        const int e = rb - S.b0[idx];  // row rb relative to the footprint's first row
                        if (e >= NB || e <= -4) continue;
                        const float wu = S.Fu[d][idx];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int er = e + r;
                            if (er >= 0 && er < NB) acc[r] = fmaf(wu, S.Fv[er][idx], acc[r]);
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
        if (b < g.nv)
            st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a,
                   DD ? acc[r] * dd_len<false>(V, g, a, b) : acc[r], out_t);
    }
}

// ------------------------------------------------------------ launchers
namespace {
template <typename TIn, bool DD, int NA, int NB>
cudaError_t nc_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out, int out_t,
                        int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (dir == 0) {
        const int tiles_u = (g.nu + 15) / 16, tiles_v = (g.nv + 63) / 64;
        dim3 blk(16, 16), grd((unsigned)((size_t)tiles_u * tiles_v * g.nview * batch));
        nc_fwd<TIn, DD, NA, NB><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u, tiles_v);
    } else {
        constexpr int ZT = 8;
        const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + ZT - 1) / ZT;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        nc_back<TIn, DD, NA, NB, ZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
    }
    return cudaGetLastError();
}

template <typename TIn, bool DD, int NA>
cudaError_t nc_rows(int dir, const CtGrid &g, const CtView *views, const void *in, void *out, int out_t,
                    int batch, cudaStream_t st) {
    // an axial rectangle of half height m rows meets at most 3 rows when
    // m <= 1 and at most 4 when m <= 1.5
    return g.max_m_sf_v <= 1.0f ? nc_launch_t<TIn, DD, NA, 3>(dir, g, views, in, out, out_t, batch, st)
                                : nc_launch_t<TIn, DD, NA, 4>(dir, g, views, in, out, out_t, batch, st);
}

// a trapezoid of half width m cells meets at most 4 cells when m <= 1.5,
// 6 when m <= 2.5 and 8 when m <= 3.5
template <typename TIn, bool DD>
cudaError_t nc_cells(int dir, const CtGrid &g, const CtView *views, const void *in, void *out, int out_t,
                     int batch, cudaStream_t st) {
    const float m = DD ? g.max_m_dd_u : g.max_m_sf_u;
    if (m <= 1.5f) return nc_rows<TIn, DD, 4>(dir, g, views, in, out, out_t, batch, st);
    if (m <= 2.5f) return nc_rows<TIn, DD, 6>(dir, g, views, in, out, out_t, batch, st);
    return nc_rows<TIn, DD, 8>(dir, g, views, in, out, out_t, batch, st);
}
}  // namespace

bool nc_footprint_fits(const CtGrid &g, int dd) {
    // at most 8 cells (half width <= 3.5) by 4 rows (half height <= 1.5)
    return (dd ? g.max_m_dd_u : g.max_m_sf_u) <= 3.5f && g.max_m_sf_v <= 1.5f;
}

cudaError_t launch_nc(int dd, int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0:
        return dd ? nc_cells<float, true>(dir, g, views, in, out, out_t, batch, st)
                  : nc_cells<float, false>(dir, g, views, in, out, out_t, batch, st);
    case 1:
        return dd ? nc_cells<__half, true>(dir, g, views, in, out, out_t, batch, st)
                  : nc_cells<__half, false>(dir, g, views, in, out, out_t, batch, st);
    default:
        return dd ? nc_cells<__nv_bfloat16, true>(dir, g, views, in, out, out_t, batch, st)
                  : nc_cells<__nv_bfloat16, false>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
