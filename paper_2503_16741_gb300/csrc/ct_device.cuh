// ct_device.cuh -- device helpers shared by the projector kernels: storage
// conversion, detector mapping in local (cell-relative) coordinates, the SF
// trapezoid integral, interval overlaps and the forward-gather search.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "ct_types.h"

namespace ctp {

// ---------------------------------------------------------------- storage
template <typename T> __device__ __forceinline__ float ld(const T *__restrict__ p, size_t i);
template <> __device__ __forceinline__ float ld<float>(const float *__restrict__ p, size_t i) {
    return __ldg(p + i);
}
template <> __device__ __forceinline__ float ld<__half>(const __half *__restrict__ p, size_t i) {
    return __half2float(__ldg(p + i));
}
template <> __device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16 *__restrict__ p,
                                                               size_t i) {
    return __bfloat162float(__ldg(p + i));
}

// four consecutive elements from an address aligned to 4 elements
__device__ __forceinline__ void ld4(const float *__restrict__ p, float v[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const __half *__restrict__ p, float v[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ld4(const __nv_bfloat16 *__restrict__ p, float v[4]) {
    const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&q.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// eight consecutive elements from an address aligned to 8 elements (one
// 32-byte sector of FP32, one 16-byte load of FP16 / BF16)
__device__ __forceinline__ void ld8(const float *__restrict__ p, float v[8]) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(__cvta_generic_to_global(p)));
}
__device__ __forceinline__ void ld8(const __half *__restrict__ p, float v[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
    const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[t]));
        v[2 * t] = f.x;
        v[2 * t + 1] = f.y;
    }
}
__device__ __forceinline__ void ld8(const __nv_bfloat16 *__restrict__ p, float v[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
    const unsigned w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[t]));
        v[2 * t] = f.x;
        v[2 * t + 1] = f.y;
    }
}

// out_t: 0 = f32, 1 = f16, 2 = bf16; one rounding at the store
__device__ __forceinline__ void st(void *out, size_t i, float v, int out_t) {
    if (out_t == 0)
        static_cast<float *>(out)[i] = v;
    else if (out_t == 1)
        static_cast<__half *>(out)[i] = __float2half_rn(v);
    else
        static_cast<__nv_bfloat16 *>(out)[i] = __float2bfloat16_rn(v);
}

// plain (coherent) loads of the output buffer for the accumulate epilogue
__device__ __forceinline__ float ldo_f(const void *p, size_t i, int t) {
    if (t == 0) return static_cast<const float *>(p)[i];
    if (t == 1) return __half2float(static_cast<const __half *>(p)[i]);
    return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[i]);
}
// Output epilogue: out = alpha * value + beta * out (beta = 0: out is only
// written; alpha = 1, beta = 0 stores the value unchanged).  Each element is
// read and written by the thread that produced it, so out may be updated in
// place.
__device__ __forceinline__ void st_out(const CtGrid &g, void *out, size_t i, float v, int out_t) {
    float r = g.alpha * v;
    if (g.beta != 0.f) r = fmaf(g.beta, ldo_f(out, i, out_t), r);
    st(out, i, r, out_t);
}

// ---------------------------------------------------------------- intervals
__device__ __forceinline__ float overlap(float lo1, float hi1, float lo2, float hi2) {
    return fmaxf(fminf(hi1, hi2) - fmaxf(lo1, lo2), 0.f);
}

// Integral from -inf to x of the unit ramp that rises from 0 at 0 to 1 at e
// and stays 1 after it; e = 0 is the unit step.  No division by a vanishing e.
__device__ __forceinline__ float ramp_int(float x, float e) {
    float xc = fminf(fmaxf(x, 0.f), e);
    return fmaf(xc * xc, 0.5f / fmaxf(e, 1e-30f), fmaxf(x - e, 0.f));
}

// same with the factor 0.5 / max(e, tiny) supplied by the caller
__device__ __forceinline__ float ramp_int_h(float x, float e, float half_inv_e) {
    float xc = fminf(fmaxf(x, 0.f), e);
    return fmaf(xc * xc, half_inv_e, fmaxf(x - e, 0.f));
}

// Unit-height trapezoid with knots k0 <= k1 <= k2 <= k3 (cell units), and
// its integral over cell [d - 1/2, d + 1/2]: the SF transaxial weight.
// h1, h3 = 0.5 / (rise width), 0.5 / (fall width), formed once per trapezoid.
struct Trap {
    float k0, k1, k2, k3;
    float h1, h3;
};
// (fast reciprocals: a ramp's slope factor carries ~2 ulp, ~1e-7 of its weights)
__device__ __forceinline__ Trap make_trap(float k0, float k1, float k2, float k3) {
    return Trap{k0, k1, k2, k3, __fdividef(0.5f, fmaxf(k1 - k0, 1e-30f)), __fdividef(0.5f, fmaxf(k3 - k2, 1e-30f))};
}
__device__ __forceinline__ float trap_G(const Trap &t, float u) {
    return ramp_int_h(u - t.k0, t.k1 - t.k0, t.h1) - ramp_int_h(u - t.k2, t.k3 - t.k2, t.h3);
}
__device__ __forceinline__ float trap_cell(const Trap &t, int d) {
    float u = (float)d;
    return trap_G(t, u + 0.5f) - trap_G(t, u - 0.5f);
}
// trapezoid weights of the 4 cells d0 .. d0+3 (zero past d1), sharing the
// antiderivative at their common edges; each equals trap_cell(t, d0 + q)
__device__ __forceinline__ void trap_cells4(const Trap &t, int d0, int d1, float F[4]) {
    float G[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) G[q] = trap_G(t, (float)(d0 + q) - 0.5f);
#pragma unroll
    for (int q = 0; q < 4; ++q) F[q] = (d0 + q <= d1) ? G[q + 1] - G[q] : 0.f;
}

// weights of the N cells d0 .. d0+N-1 (zero past d1); each equals trap_cell
template <int N>
__device__ __forceinline__ void trap_cellsN(const Trap &t, int d0, int d1, float F[N]) {
    float Gp = trap_G(t, (float)d0 - 0.5f);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const float Gn = trap_G(t, (float)(d0 + q) + 0.5f);
        F[q] = (d0 + q <= d1) ? Gn - Gp : 0.f;
        Gp = Gn;
    }
}

// Axial rectangle [lo, hi] of width < 1 row (relative to a row grid whose
// row e covers [e - 1/2, e + 1/2]): it meets rows e0 and e0 + 1 only, with
// the overlaps below (equal to overlap(lo, hi, e -+ 1/2) bit for bit).
__device__ __forceinline__ void two_rows(float lo, float hi, int &e0, float &F0, float &F1) {
    const float ef = floorf(lo + 0.5f);
    e0 = (int)ef;
    const float m = ef + 0.5f;
    F0 = fmaxf(fminf(hi, m) - fmaxf(lo, ef - 0.5f), 0.f);
    F1 = fmaxf(hi - m, 0.f);
}

__device__ __forceinline__ void cswap(float &a, float &b) {
    float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}
__device__ __forceinline__ void sort4(float &a, float &b, float &c, float &d) {
    cswap(a, b);
    cswap(c, d);
    cswap(a, c);
    cswap(b, d);
    cswap(b, c);
}

// ---------------------------------------------------------------- detector map
// (a, b, c) = (w.e_u, w.n, w.e_v) of a point; fractional cell coordinates.
template <bool CURVED> struct Det {
    __device__ static __forceinline__ float fu(const CtView &V, float a, float b) {
        return CURVED ? fmaf(V.Ku, atan2f(a, b), V.Cu) : fmaf(V.Ku, a / b, V.Cu);
    }
    // "depth" that divides w.e_v: w.n (flat) or the distance from the source axis (curved)
    __device__ static __forceinline__ float den(float a, float b) {
        return CURVED ? sqrtf(fmaf(a, a, b * b)) : b;
    }
    // fu(a + da, b + db) - fu(a, b), formed from the small offsets directly
    // (a difference of about one cell: the fast division's 2 ulp are ~1e-7 cell)
    __device__ static __forceinline__ float dfu(const CtView &V, float a, float b, float da, float db) {
        float num = fmaf(da, b, -a * db);
        if (CURVED) return V.Ku * atan2f(num, fmaf(a + da, a, (b + db) * b));
        return V.Ku * __fdividef(num, (b + db) * b);
    }
    // ratio (w.e_u)/(w.n) at which fu equals F (for the forward search planes)
    __device__ static __forceinline__ float ratio_at(const CtView &V, float F) {
        float t = (F - V.Cu) / V.Ku;
        return CURVED ? tanf(t) : t;
    }
};

// nearest cell to a fractional coordinate, and the remainder in [-1/2, 1/2)
__device__ __forceinline__ void split_cell(float f, int &ref, float &frac) {
    float r = floorf(f + 0.5f);
    ref = (int)r;
    frac = f - r;
}

// DD path length of cell (a, b): slab width times |d| / |d_main| of the ray
// from the source to the cell centre (d in world coordinates).
template <bool CURVED>
__device__ __forceinline__ float dd_len(const CtView &V, const CtGrid &g, int a, int b) {
    const float Vb = g.dv * ((float)b - V.Cv);
    float d2, dm;
    const int m = V.main_y;
    const float nm = m ? V.nn[1] : V.nn[0];
    const float um = m ? V.eu[1] : V.eu[0];
    const float vm = m ? V.ev[1] : V.ev[0];
    if (CURVED) {
        float sg, cg;
        sincosf(((float)a - V.Cu) / V.Ku, &sg, &cg);
        d2 = fmaf(V.D, V.D, Vb * Vb);
        dm = fmaf(V.D, fmaf(cg, nm, sg * um), Vb * vm);
    } else {
        const float U = g.du * ((float)a - V.Cu);
        d2 = fmaf(V.D, V.D, fmaf(U, U, Vb * Vb));
        dm = fmaf(V.D, nm, fmaf(U, um, Vb * vm));
    }
    return (m ? g.dy : g.dx) * sqrtf(d2) / fabsf(dm);
}

// SF-TT amplitude ("A2") of cell (a, b) on a flat detector: the SF-TR
// amplitude taken along the ray to the cell centre, dx |d| / max(|d_x|, |d_y|)
// with d = (cell centre - source) in world coordinates.
__device__ __forceinline__ float tt_amp(const CtView &V, const CtGrid &g, int a, int b) {
    const float U = g.du * ((float)a - V.Cu), Vb = g.dv * ((float)b - V.Cv);
    const float dx_ = fmaf(V.D, V.nn[0], fmaf(U, V.eu[0], Vb * V.ev[0]));
    const float dy_ = fmaf(V.D, V.nn[1], fmaf(U, V.eu[1], Vb * V.ev[1]));
    const float dz_ = fmaf(V.D, V.nn[2], fmaf(U, V.eu[2], Vb * V.ev[2]));
    return g.dx * sqrtf(fmaf(dx_, dx_, fmaf(dy_, dy_, dz_ * dz_))) / fmaxf(fabsf(dx_), fabsf(dy_));
}

// ---------------------------------------------------------------- forward search
// Candidate lateral/axial index box of slab s for the detector window
// fu in [Flo, Fhi], fv in [Glo, Ghi] of a flat detector: the window's four
// corner rays cut the slab plane in a quadrilateral whose bounding box holds
// every voxel centre that projects into the window.
struct SlabCoef {
    float ul, uk, us, u3;  // au along (lateral, k, slab, const)
    float nl, nk, ns, n3;  // an
    float vl, vk, vs, v3;  // av
};
__device__ __forceinline__ SlabCoef slab_coef(const CtView &V, int main_y) {
    SlabCoef c;
    if (main_y) {
        c.ul = V.au[0]; c.us = V.au[1];
        c.nl = V.an[0]; c.ns = V.an[1];
        c.vl = V.av[0]; c.vs = V.av[1];
    } else {
        c.ul = V.au[1]; c.us = V.au[0];
        c.nl = V.an[1]; c.ns = V.an[0];
        c.vl = V.av[1]; c.vs = V.av[0];
    }
    c.uk = V.au[2]; c.u3 = V.au[3];
    c.nk = V.an[2]; c.n3 = V.an[3];
    c.vk = V.av[2]; c.v3 = V.av[3];
    return c;
}

// Flat detector: corners of {Ku au - (F-Cu) an = 0} x {Kv av - (G-Cv) an = 0}
__device__ __forceinline__ bool search_flat(const CtView &V, const SlabCoef &c, int s, float Flo,
                                            float Fhi, float Glo, float Ghi, int nlat, int nk,
                                            int &l0, int &l1, int &k0, int &k1) {
    float lmin = 3.0e38f, lmax = -3.0e38f, kmin = 3.0e38f, kmax = -3.0e38f;
    float fs = (float)s;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float tu = (q ? Fhi : Flo) - V.Cu;
        float Pl = fmaf(V.Ku, c.ul, -tu * c.nl);
        float Pk = fmaf(V.Ku, c.uk, -tu * c.nk);
        float Pc = fmaf(V.Ku, fmaf(c.us, fs, c.u3), -tu * fmaf(c.ns, fs, c.n3));
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            float tv = (r ? Ghi : Glo) - V.Cv;
            float Ql = fmaf(V.Kv, c.vl, -tv * c.nl);
            float Qk = fmaf(V.Kv, c.vk, -tv * c.nk);
            float Qc = fmaf(V.Kv, fmaf(c.vs, fs, c.v3), -tv * fmaf(c.ns, fs, c.n3));
            float det = fmaf(Pl, Qk, -Pk * Ql);
            float l = fmaf(-Pc, Qk, Qc * Pk) / det;
            float k = fmaf(-Qc, Pl, Pc * Ql) / det;
            lmin = fminf(lmin, l); lmax = fmaxf(lmax, l);
            kmin = fminf(kmin, k); kmax = fmaxf(kmax, k);
        }
    }
    l0 = max(0, (int)ceilf(lmin));
    l1 = min(nlat - 1, (int)floorf(lmax));
    k0 = max(0, (int)ceilf(kmin));
    k1 = min(nk - 1, (int)floorf(kmax));
    return l0 <= l1 && k0 <= k1 && isfinite(lmin) && isfinite(lmax);
}

// Circular geometry (e_v = z, e_u and n horizontal): the u window is cut by
// two vertical planes through the source axis; the v window by two planes
// (flat) or cones (curved) through the source, bounded with the extreme
// depths of the candidate columns.
template <bool CURVED>
__device__ __forceinline__ bool search_circ(const CtView &V, const SlabCoef &c, int s, float Flo,
                                            float Fhi, float Glo, float Ghi, int nlat, int nk,
                                            int &l0, int &l1, int &k0, int &k1) {
    const float fs = (float)s;
    const float Bu = fmaf(c.us, fs, c.u3), Bn = fmaf(c.ns, fs, c.n3);
    const float T1 = Det<CURVED>::ratio_at(V, Flo), T2 = Det<CURVED>::ratio_at(V, Fhi);
    const float la = (T1 * Bn - Bu) / (c.ul - T1 * c.nl);
    const float lb = (T2 * Bn - Bu) / (c.ul - T2 * c.nl);
    l0 = max(0, (int)ceilf(fminf(la, lb)));
    l1 = min(nlat - 1, (int)floorf(fmaxf(la, lb)));
    if (l0 > l1) return false;
    const float fl0 = (float)l0, fl1 = (float)l1;
    const float b0 = fmaf(c.nl, fl0, Bn), b1 = fmaf(c.nl, fl1, Bn);
    float rmin, rmax;
    if (CURVED) {
        const float a0 = fmaf(c.ul, fl0, Bu), a1 = fmaf(c.ul, fl1, Bu);
        const float r0 = sqrtf(fmaf(a0, a0, b0 * b0)), r1 = sqrtf(fmaf(a1, a1, b1 * b1));
        rmax = fmaxf(r0, r1);
        rmin = fminf(r0, r1);
        const float g2 = fmaf(c.ul, c.ul, c.nl * c.nl);
        const float ls = -fmaf(c.ul, Bu, c.nl * Bn) / g2;  // closest approach to the axis
        if (ls > fl0 && ls < fl1) {
            const float as = fmaf(c.ul, ls, Bu), bs = fmaf(c.nl, ls, Bn);
            rmin = sqrtf(fmaf(as, as, bs * bs));
        }
    } else {
        rmin = fminf(b0, b1);
        rmax = fmaxf(b0, b1);
    }
    rmin *= 0.9999f;  // rounding guard on the bound
    rmax *= 1.0001f;
    const float tlo = (Glo - V.Cv) / V.Kv, thi = (Ghi - V.Cv) / V.Kv;
    const float cmin = fminf(tlo * rmin, tlo * rmax), cmax = fmaxf(thi * rmin, thi * rmax);
    // w.e_v = vk k + v3 (e_v = z: no lateral or slab term)
    const float ka = (cmin - c.v3) / c.vk, kb = (cmax - c.v3) / c.vk;
    k0 = max(0, (int)ceilf(fminf(ka, kb)));
    k1 = min(nk - 1, (int)floorf(fmaxf(ka, kb)));
    return k0 <= k1;
}

template <bool CURVED>
__device__ __forceinline__ bool slab_search(const CtView &V, const SlabCoef &c, int s, float Flo,
                                            float Fhi, float Glo, float Ghi, int nlat, int nk,
                                            int &l0, int &l1, int &k0, int &k1) {
    return search_circ<CURVED>(V, c, s, Flo, Fhi, Glo, Ghi, nlat, nk, l0, l1, k0, k1);
}

// ---------------------------------------------------------------- voxel-driven
// Voxel-driven amplitude (Peters 1981, cited in Sec. 2.3): the voxel's mass
// spread over the local ray density,
//   3D  A = dx dy dz r D^2 / (rho^3 du dv)      2D  A = dx dy r D / (rho^2 du)
// with r = |X - s| and rho the depth (flat) or distance from the source axis
// (curved).
__device__ __forceinline__ float vx_amp(const CtGrid &g, const CtView &V, float r, float den) {
    if (g.is2d) return (g.dx * g.dy / g.du) * r * V.D / (den * den);
    const float q = V.D / den;
    return (g.dx * g.dy * g.dz / (g.du * g.dv)) * (r / den) * q * q;
}

// circular geometry: column quantities shared down z
struct VxCol {
    float fu;         // fractional u of the column (all z)
    float sv, fv0;    // fv of voxel k: sv * k + fv0
    float rxy2, den;  // w_x^2 + w_y^2 and the depth rho
    float amp1;       // amplitude per unit r: A = amp1 r
};

template <bool CURVED>
__device__ __forceinline__ VxCol vx_col(const CtView &V, const CtGrid &g, int i, int j) {
    const float fi = (float)i, fj = (float)j;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, V.au[3]));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, V.an[3]));
    VxCol C;
    C.fu = Det<CURVED>::fu(V, cu, cn);
    C.den = Det<CURVED>::den(cu, cn);
    C.sv = V.Kv * V.av[2] / C.den;
    C.fv0 = fmaf(V.Kv, V.av[3] / C.den, V.Cv);
    const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
    C.rxy2 = fmaf(wx, wx, wy * wy);
    C.amp1 = vx_amp(g, V, 1.f, C.den);
    return C;
}

__device__ __forceinline__ float vx_amp_col(const VxCol &C, const CtGrid &g, const CtView &V, int k) {
    const float wz = fmaf((float)k, g.dz, V.o[2]);
    const float t = fmaf(wz, wz, C.rxy2);
    return C.amp1 * (t * rsqrtf(t));
}

// rounding guard added to every search window (cells)
constexpr float kSearchPad = 2e-3f;

}  // namespace ctp
