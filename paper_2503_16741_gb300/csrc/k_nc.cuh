// k_nc.cuh -- SF-TR and DD footprint projectors in non-circular geometry
// (flat detector with per-view tilt and in-plane rotation, Sec. 2.2), where a
// voxel's transaxial footprint changes with its z (the footprint methods cited
// in Sec. 2.3: Long, Fessler & Balter 2010; De Man & Basu 2004), and the
// SF-TT projector (trapezoid x trapezoid, per-cell amplitude; the same
// paper's variant for large cone angles) on any flat detector.  Every voxel
// carries its own footprint of at most NA cells by NB rows (NA = 4, 6 or 8,
// NB = 3 or 4, chosen by the launcher from the per-view footprint bounds;
// wider footprints go to the general kernels).
//   back:    thread = voxel column over a z-chunk, all views (records staged
//            in shared memory); per voxel and view the footprint, then its
//            NA x NB taps.
//   forward: CTA = 64 cells x 64 rows of one view.  Per slab of the view's
//            main axis the CTA computes, once, the footprint of every voxel
//            that can reach its tile into shared memory (a footprint cache);
//            each thread then gathers, for its 4 cells x 4 rows, the cached
//            weights of the voxels in its own search box.
// Both are gathers with a fixed summation order: deterministic, no atomics.
// DD and SF-TT multiply by their per-cell factor (path length L_c, amplitude
// A2) after the forward gather; their back direction takes a sinogram already
// scaled by it.
// This header holds the per-voxel footprint both directions evaluate and the
// dispatch over footprint sizes; the kernels are in k_nc_fwd.cu and
// k_nc_back.cu.
#pragma once
#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {


// projector kinds of these kernels
enum NcKind { NC_SF = 0, NC_DD = 1, NC_TT = 2 };

template <int NA, int NB> struct NcFp {
    int a0, b0;    // first cell, first row of the footprint
    int n;         // cells with a weight (at most NA)
    float Fu[NA];  // transaxial weights of cells a0 .. a0 + NA - 1
    float Fv[NB];  // axial weights of rows b0 .. b0 + NB - 1
    float amp;     // SF-TR amplitude dx |w| / max(|w_x|, |w_y|); DD, SF-TT: 1 (their factor is per cell)
    float cn;      // depth (X - s).n of the voxel centre
    float size;    // SF-TR, DD: transaxial area (cells) x axial height (rows) of the footprint
};

// Trapezoid with the ramp factors formed by a fast reciprocal (relative
// error ~1e-7 on a ramp's slope).
__device__ __forceinline__ Trap nc_trap(float k0, float k1, float k2, float k3) {
    return Trap{k0, k1, k2, k3, __fdividef(0.5f, fmaxf(k1 - k0, 1e-30f)), __fdividef(0.5f, fmaxf(k3 - k2, 1e-30f))};
}

// Weights of the cells d0 .. d1 (at most N) under trapezoid T, from its
// antiderivative G at their edges: G = 0 at the first edge (left of k0) and
// the trapezoid's area at the last (right of k3), so only the interior edges
// are evaluated.  A footprint wider than the bound by rounding loses the
// cells past N - 1, whose weight is of the order of the rounding.  Returns
// the count of cells with a weight.
template <int N>
__device__ __forceinline__ int nc_cells(const Trap &T, int d0, int d1, float (&F)[N]) {
#pragma unroll
    for (int q = 0; q < N; ++q) F[q] = 0.f;
    const int nlast = d1 - d0;  // index of the last cell
    const float e0 = (float)d0 + 0.5f;  // right edge of the first cell (exact)
    float Gp = 0.f;
#pragma unroll
    for (int q = 0; q < N - 1; ++q) {
        if (q >= nlast) break;
        const float Gn = trap_G(T, e0 + (float)q);
        F[q] = Gn - Gp;
        Gp = Gn;
    }
    float Glast = 0.5f * ((T.k3 - T.k0) + (T.k2 - T.k1));
    if (nlast >= N) Glast = trap_G(T, (float)(d0 + N - 1) + 0.5f);
    const int ql = min(nlast, N - 1);
#pragma unroll
    for (int q = 0; q < N; ++q)
        if (q == ql) F[q] = Glast - Gp;
    return ql + 1;
}

// Footprint of voxel (i, j, k) in view V.  The centre is projected with a
// correctly rounded reciprocal; corner and end-point offsets are formed from
// small differences, K (du - r dn) / (cn + dn) with r = cu / cn, where a fast
// division's few ulp are ~1e-7 cell.
//   SF-TR: trapezoid from the four transaxial corners x rectangle from the
//          z ends at the (x, y) centre, voxel amplitude;
//   DD:    box between the lateral boundary points x the same rectangle;
//   SF-TT: the SF-TR trapezoid x a trapezoid from the z faces at the
//          transaxial corners nearest to and farthest from the source
//          (against the normal's transaxial components; a component below
//          1e-7 of the voxel size counts as zero and takes the negative
//          side), amplitude per cell.
template <int KIND, int NA, int NB>
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
    if (KIND == NC_DD) {  // boundary points +- half a voxel along the lateral axis
        const int q = V.main_y ? 0 : 1;
        const float hu = 0.5f * V.au[q], hn = 0.5f * V.an[q];
        const float e1 = fr + V.Ku * __fdividef(fmaf(r, hn, -hu), cn - hn);
        const float e2 = fr + V.Ku * __fdividef(fmaf(-r, hn, hu), cn + hn);
        const float lo = fminf(e1, e2), hi = fmaxf(e1, e2);
        T = nc_trap(lo, lo, hi, hi);
    } else {  // the four transaxial corners, sorted into a trapezoid
        float t0 = fr + V.Ku * __fdividef(fmaf(-r, V.cdn[0], V.cdu[0]), cn + V.cdn[0]);
        float t1 = fr + V.Ku * __fdividef(fmaf(-r, V.cdn[1], V.cdu[1]), cn + V.cdn[1]);
        float t2 = fr + V.Ku * __fdividef(fmaf(-r, V.cdn[2], V.cdu[2]), cn + V.cdn[2]);
        float t3 = fr + V.Ku * __fdividef(fmaf(-r, V.cdn[3], V.cdu[3]), cn + V.cdn[3]);
        sort4(t0, t1, t2, t3);
        T = nc_trap(t0, t1, t2, t3);
    }
    const int d0 = (int)floorf(T.k0 + 0.5f), d1 = (int)floorf(T.k3 + 0.5f);
    P.n = nc_cells<NA>(T, d0, d1, P.Fu);
    P.a0 = aref + d0;
    const float hzv = V.hzv, hzn = V.hzn;
    if (KIND == NC_TT) {
        if (g.is2d) {  // one row of unit height, inside the axial plateau: factor 1
#pragma unroll
            for (int q = 0; q < NB; ++q) P.Fv[q] = q == 0 ? 1.f : 0.f;
            P.b0 = 0;
        } else {
            const float eps = 1e-7f * g.dx;
            const float hxn = 0.5f * V.an[0], hyn = 0.5f * V.an[1];
            const float hxv = 0.5f * V.av[0], hyv = 0.5f * V.av[1];
            const float snx = V.an[0] < -eps ? 1.f : -1.f, sny = V.an[1] < -eps ? 1.f : -1.f;  // nearest
            const float sfx = V.an[0] > eps ? 1.f : -1.f, sfy = V.an[1] > eps ? 1.f : -1.f;    // farthest
            const float nv_ = fmaf(snx, hxv, sny * hyv), nn_ = fmaf(snx, hxn, sny * hyn);
            const float fv_ = fmaf(sfx, hxv, sfy * hyv), fn_ = fmaf(sfx, hxn, sfy * hyn);
            float t0 = vr + V.Kv * __fdividef(fmaf(-rv, nn_ - hzn, nv_ - hzv), cn + nn_ - hzn);
            float t1 = vr + V.Kv * __fdividef(fmaf(-rv, nn_ + hzn, nv_ + hzv), cn + nn_ + hzn);
            float t2 = vr + V.Kv * __fdividef(fmaf(-rv, fn_ - hzn, fv_ - hzv), cn + fn_ - hzn);
            float t3 = vr + V.Kv * __fdividef(fmaf(-rv, fn_ + hzn, fv_ + hzv), cn + fn_ + hzn);
            sort4(t0, t1, t2, t3);
            const Trap Tv = nc_trap(t0, t1, t2, t3);
            const int e0 = (int)floorf(Tv.k0 + 0.5f), e1 = (int)floorf(Tv.k3 + 0.5f);
            nc_cells<NB>(Tv, e0, e1, P.Fv);
            P.b0 = bref + e0;
        }
    } else {  // axial rectangle: the end points (z -+ dz/2) at the voxel's (x, y) centre
        const float f1 = vr + V.Kv * __fdividef(fmaf(-rv, hzn, hzv), cn + hzn);
        const float f2 = vr + V.Kv * __fdividef(fmaf(rv, hzn, -hzv), cn - hzn);
        const float vlo = fminf(f1, f2), vhi = fmaxf(f1, f2);
        // overlaps with rows e0 .. e0 + NB - 1 (row e covers [e - 1/2, e + 1/2]);
        // vlo lies below the first row's upper edge m, so each later row's
        // overlap starts at its lower edge (equal to overlap() bit for bit)
        const float ef = floorf(vlo + 0.5f);
        float m = ef + 0.5f;
        P.Fv[0] = fmaxf(fminf(vhi, m) - fmaxf(vlo, m - 1.f), 0.f);
#pragma unroll
        for (int q = 1; q < NB; ++q) {
            P.Fv[q] = fmaxf(fminf(vhi, m + 1.f) - m, 0.f);
            m += 1.f;
        }
        P.b0 = bref + (int)ef;
        P.size = 0.5f * ((T.k3 - T.k0) + (T.k2 - T.k1)) * (vhi - vlo);
    }
    P.cn = cn;
    if (KIND != NC_SF) {
        P.amp = 1.f;
    } else {
        const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
        const float wz = fmaf(fk, g.dz, V.o[2]);
        const float t = fmaf(wx, wx, fmaf(wy, wy, wz * wz));
        P.amp = __fdividef(g.dx * t * rsqrtf(t), fmaxf(fabsf(wx), fabsf(wy)));
    }
}

// the per-cell factor of DD (path length L_c) and SF-TT (amplitude A2)
template <int KIND>
__device__ __forceinline__ float nc_cell_factor(const CtView &V, const CtGrid &g, int a, int b) {
    return KIND == NC_DD ? dd_len<false>(V, g, a, b) : tt_amp(V, g, a, b);
}

// Runs Run<TIn, KIND, NA, NB>::go(g, args...) for the storage type, the
// projector and the footprint bounds of g: a trapezoid of half width m cells
// meets at most 4 cells when m <= 1.5, 6 when m <= 2.5 and 8 when m <= 3.5;
// an axial footprint of half height m rows at most 3 rows when m <= 1 and 4
// when m <= 1.5.
template <template <typename, int, int, int> class Run, typename TIn, int KIND, typename... A>
cudaError_t nc_dispatch_t(const CtGrid &g, A... args) {
    const float m = KIND == NC_DD ? g.max_m_dd_u : g.max_m_sf_u;
    const bool r3 = (KIND == NC_TT ? g.max_m_tt_v : g.max_m_sf_v) <= 1.0f;
    if (m <= 1.5f) return r3 ? Run<TIn, KIND, 4, 3>::go(g, args...) : Run<TIn, KIND, 4, 4>::go(g, args...);
    if (m <= 2.5f) return r3 ? Run<TIn, KIND, 6, 3>::go(g, args...) : Run<TIn, KIND, 6, 4>::go(g, args...);
    return r3 ? Run<TIn, KIND, 8, 3>::go(g, args...) : Run<TIn, KIND, 8, 4>::go(g, args...);
}

template <template <typename, int, int, int> class Run, typename TIn, typename... A>
cudaError_t nc_dispatch_k(int kind, const CtGrid &g, A... args) {
    switch (kind) {
    case NC_SF: return nc_dispatch_t<Run, TIn, NC_SF>(g, args...);
    case NC_DD: return nc_dispatch_t<Run, TIn, NC_DD>(g, args...);
    default: return nc_dispatch_t<Run, TIn, NC_TT>(g, args...);
    }
}

template <template <typename, int, int, int> class Run, typename... A>
cudaError_t nc_dispatch(int kind, int in_t, const CtGrid &g, A... args) {
    switch (in_t) {
    case 0: return nc_dispatch_k<Run, float>(kind, g, args...);
    case 1: return nc_dispatch_k<Run, __half>(kind, g, args...);
    default: return nc_dispatch_k<Run, __nv_bfloat16>(kind, g, args...);
    }
}

// the two directions (k_nc_fwd.cu, k_nc_back.cu); kind: NcKind
cudaError_t launch_nc_fwd(int kind, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                          void *out, int batch, cudaStream_t st);
cudaError_t launch_nc_back(int kind, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                           void *out, int batch, cudaStream_t st);

}  // namespace ctp
