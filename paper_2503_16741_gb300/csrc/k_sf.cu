// k_sf.cu -- footprint projectors in circular geometry, and the SF-TR
// projector in non-circular geometry.
// SF-TR (Long, Fessler & Balter 2010, cited in Sec. 2.3): trapezoid
// transaxial footprint from the four projected column corners, rectangle
// axial footprint from the projected end points, amplitude dx / max(|cos|,
// |sin|) of the 3D ray to the voxel centre.
// DD (De Man & Basu 2004, cited in Sec. 2.3) in circular geometry shares the
// kernels: its transaxial footprint is the box between the two projected
// boundary points (a trapezoid with vertical sides), its axial footprint the
// same rectangle, its amplitude 1, and each cell carries the path length L_c
// of its central ray through one slab -- applied once per cell after the
// gather in the forward, and to the sinogram before the gather in the back.
// Forward and back are gather kernels (no atomics) that evaluate the same
// per-voxel weight functions, so they form a matched pair.  The streaming
// forward also serves the voxel-driven projector in circular geometry (its
// hat weights in place of the footprints; the back kernel is in k_voxel.cu).
#include <algorithm>

#include "ct_device.cuh"
#include "ct_launch.h"
#include "k_nc.cuh"

namespace ctp {

// ------------------------------------------------------------ weights
// Circular geometry: the transaxial footprint of column (i, j) does not
// depend on z, so it is computed once per (column, view) and reused down z.
struct SfCol {
    Trap T;        // knots relative to cell aref (cell units)
    int aref;
    float sv, fv0; // fv of voxel centre k: sv * k + fv0
    float hv;      // half height of the axial rectangle (rows)
    float invm;    // dx / max(|w_x|, |w_y|)
    float rxy2;    // w_x^2 + w_y^2
};

template <bool CURVED, bool DD = false>
__device__ __forceinline__ SfCol sf_col(const CtView &V, const CtGrid &g, int i, int j) {
    const float fi = (float)i, fj = (float)j;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, V.au[3]));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, V.an[3]));
    SfCol C;
    float fr;
    split_cell(Det<CURVED>::fu(V, cu, cn), C.aref, fr);
    if (DD) {
        // boundary points +- half a voxel along the non-main axis
        const int q = V.main_y ? 0 : 1;
        const float hu = 0.5f * V.au[q], hn = 0.5f * V.an[q];
        const float e1 = fr + Det<CURVED>::dfu(V, cu, cn, -hu, -hn);
        const float e2 = fr + Det<CURVED>::dfu(V, cu, cn, hu, hn);
        const float lo = fminf(e1, e2), hi = fmaxf(e1, e2);
        C.T = make_trap(lo, lo, hi, hi);
    } else {
        const float hxu = 0.5f * V.au[0], hxn = 0.5f * V.an[0];
        const float hyu = 0.5f * V.au[1], hyn = 0.5f * V.an[1];
        float t0 = fr + Det<CURVED>::dfu(V, cu, cn, -hxu - hyu, -hxn - hyn);
        float t1 = fr + Det<CURVED>::dfu(V, cu, cn, hxu - hyu, hxn - hyn);
        float t2 = fr + Det<CURVED>::dfu(V, cu, cn, -hxu + hyu, -hxn + hyn);
        float t3 = fr + Det<CURVED>::dfu(V, cu, cn, hxu + hyu, hxn + hyn);
        sort4(t0, t1, t2, t3);
        C.T = make_trap(t0, t1, t2, t3);
    }
    const float kd = V.Kv / Det<CURVED>::den(cu, cn);
    C.sv = kd * V.av[2];
    C.fv0 = fmaf(kd, V.av[3], V.Cv);
    C.hv = 0.5f * fabsf(C.sv);
    const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
    C.rxy2 = fmaf(wx, wx, wy * wy);
    C.invm = __fdividef(g.dx, fmaxf(fabsf(wx), fabsf(wy)));
    return C;
}

__device__ __forceinline__ float sf_amp(const SfCol &C, const CtGrid &g, const CtView &V, int k) {
    const float wz = fmaf((float)k, g.dz, V.o[2]);
    return C.invm * sqrtf(fmaf(wz, wz, C.rxy2));
}

// SF-TT in circular flat geometry (the transaxial footprint is SF-TR's): the
// axial trapezoid of voxel k has its knots on the z faces at the column's
// transaxial corners nearest to and farthest from the source (against the
// normal's transaxial components; a component below 1e-7 of the voxel size
// counts as zero and takes the negative side).  A corner at depth cn (1 + e)^-1
// projects the voxel's centre to fv(k) + g(k) e and its z faces to -+ hv (1 + e)
// about that, with g(k) = fv(k) - Cv = sv k + g0 linear in k.
struct TtCol {
    float g0;
    float eN, eF;  // nearest, farthest corner: cn / depth - 1
    float hN, hF;  // half heights hv (1 + e)
};

__device__ __forceinline__ TtCol tt_col(const CtView &V, const CtGrid &g, const SfCol &C, int i, int j) {
    const float cn = fmaf(V.an[0], (float)i, fmaf(V.an[1], (float)j, V.an[3]));
    const float eps = 1e-7f * g.dx;
    const float hxn = 0.5f * V.an[0], hyn = 0.5f * V.an[1];
    const float nn = (V.an[0] < -eps ? hxn : -hxn) + (V.an[1] < -eps ? hyn : -hyn);
    const float fn = (V.an[0] > eps ? hxn : -hxn) + (V.an[1] > eps ? hyn : -hyn);
    TtCol T;
    T.eN = -nn / (cn + nn);
    T.eF = -fn / (cn + fn);
    T.hN = fmaf(C.hv, T.eN, C.hv);
    T.hF = fmaf(C.hv, T.eF, C.hv);
    T.g0 = (V.Kv / cn) * V.av[3];
    return T;
}

// rows e0 .. e0 + 3 (relative to the row of the voxel centre, whose offset
// in it is vf) under the axial trapezoid of voxel fk, and their weights
// (zero past the trapezoid; it spans at most 4 rows when its half height
// bound is at most 1.5 rows)
__device__ __forceinline__ void tt_rows(const SfCol &C, const TtCol &T, float fk, float vf, int &e0,
                                        float (&Fv)[4]) {
    const float gk = fmaf(C.sv, fk, T.g0);
    const float cN = fmaf(gk, T.eN, vf), cF = fmaf(gk, T.eF, vf);
    float t0 = cN - T.hN, t1 = cN + T.hN, t2 = cF - T.hF, t3 = cF + T.hF;
    sort4(t0, t1, t2, t3);
    const Trap Tv = nc_trap(t0, t1, t2, t3);
    e0 = (int)floorf(Tv.k0 + 0.5f);
    nc_cells<4>(Tv, e0, (int)floorf(Tv.k3 + 0.5f), Fv);
}

// the 4-cell window [as, as + 3] inside the detector (nu >= 4) for the weights
// F of cells a0 .. a0 + 3: shifted when the footprint sits on the last cells
__device__ __forceinline__ int window4(const float (&F)[4], int a0, int nu, float (&Fu)[4]) {
    const int as = min(a0, nu - 4);
    const int sh = a0 - as;  // 0..3
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float w = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) w = (q - sh == p) ? F[p] : w;
        Fu[q] = w;
    }
    return as;
}

// Non-circular flat geometry: everything per voxel.
struct SfVox {
    Trap T;
    int aref, bref;
    float vlo, vhi;  // axial rectangle relative to row bref
    float amp;
};

__device__ __forceinline__ float dratio(float K, float c, float b, float dc, float db) {
    return K * fmaf(dc, b, -c * db) / ((b + db) * b);
}

__device__ __forceinline__ SfVox sf_vox_nc(const CtView &V, const CtGrid &g, int i, int j, int k) {
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, fmaf(V.au[2], fk, V.au[3])));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, fmaf(V.an[2], fk, V.an[3])));
    const float cv = fmaf(V.av[0], fi, fmaf(V.av[1], fj, fmaf(V.av[2], fk, V.av[3])));
    SfVox P;
    float fr, vr;
    split_cell(fmaf(V.Ku, cu / cn, V.Cu), P.aref, fr);
    split_cell(fmaf(V.Kv, cv / cn, V.Cv), P.bref, vr);
    const float hxu = 0.5f * V.au[0], hxn = 0.5f * V.an[0];
    const float hyu = 0.5f * V.au[1], hyn = 0.5f * V.an[1];
    float t0 = fr + dratio(V.Ku, cu, cn, -hxu - hyu, -hxn - hyn);
    float t1 = fr + dratio(V.Ku, cu, cn, hxu - hyu, hxn - hyn);
    float t2 = fr + dratio(V.Ku, cu, cn, -hxu + hyu, -hxn + hyn);
    float t3 = fr + dratio(V.Ku, cu, cn, hxu + hyu, hxn + hyn);
    sort4(t0, t1, t2, t3);
    P.T = make_trap(t0, t1, t2, t3);
    const float hzv = 0.5f * V.av[2], hzn = 0.5f * V.an[2];
    const float e1 = vr + dratio(V.Kv, cv, cn, hzv, hzn);
    const float e2 = vr + dratio(V.Kv, cv, cn, -hzv, -hzn);
    P.vlo = fminf(e1, e2);
    P.vhi = fmaxf(e1, e2);
    const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
    const float wz = fmaf(fk, g.dz, V.o[2]);
    P.amp = g.dx * sqrtf(fmaf(wx, wx, fmaf(wy, wy, wz * wz))) / fmaxf(fabsf(wx), fabsf(wy));
    return P;
}

// ------------------------------------------------------------ back (gather)
// Thread = one voxel column (i, j) over a z-chunk of ZT voxels; loops over
// all views (records staged in shared memory, kViews at a time).
// Common case (footprint <= 4 cells, axial rectangle shorter than a row):
// the column's 4 transaxial weights filter each detector row the chunk
// touches once, R(b) = sum_q Fu[q] y[b][a0 + q], into a per-thread slice of
// shared memory; each voxel then takes its two rows, x += amp (Fv0 R(b0) +
// Fv1 R(b0 + 1)).  Other footprints take the general loops.  Both evaluate
// the same weights as the forward kernel.
constexpr int kViews = 64;

__device__ __forceinline__ void stage_views(CtView *dst, const CtView *__restrict__ src, int n, int tid,
                                            int nthr) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    constexpr int W = sizeof(CtView) / sizeof(float4);
    for (int t = tid; t < n * W; t += nthr) d4[t] = __ldg(s4 + t);
}

__device__ __forceinline__ float sf_amp_fast(float invm, float rxy2, float wz) {
    const float t = fmaf(wz, wz, rxy2);
    return invm * t * rsqrtf(t);
}
// per-voxel amplitude: SF as above, DD 1 (its factor is per cell)
template <bool DD, typename C_>
__device__ __forceinline__ float fp_amp(const C_ &C, float wz) {
    return DD ? 1.f : sf_amp_fast(C.invm, C.rxy2, wz);
}

// RECON: the recon-mode (FBP) backprojection of filtered projections with the
// normalised footprints as the interpolation (Sec. 2.3): the voxel's weight
// is the depth weight rc_w / depth^2 over the footprint's transaxial area
// (cells) and axial height (rows), constant down a column.
// TT: SF-TT (flat detector), on a sinogram already scaled by the per-cell
// amplitude A2; its axial trapezoids reach further, so the row buffer holds
// ZT + 6 rows.
template <typename TIn, bool CURVED, bool DD, int ZT, bool RECON = false, bool TT = false>
__global__ void __launch_bounds__(128, ZT <= 16 ? 7 : 5)
sf_back_circ(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
             void *__restrict__ vol, int out_t, int tiles_x, int nzc) {
    constexpr int NR = TT ? ZT + 6 : ZT + 3;  // SF, DD: rows -1 .. ZT + 1 relative to the chunk's first voxel
    __shared__ CtView sview[kViews];
    __shared__ float Rs[NR][128];
    __shared__ float Gs[ZT][128];  // general-path partial sums (thread-private slots)
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool active = i < g.nx && j < g.ny;
    const int kbeg = kc * ZT;
    const int kend = min(kbeg + ZT, g.nz);
    float acc[ZT];
#pragma unroll
    for (int q = 0; q < ZT; ++q) {
        acc[q] = 0.f;
        Gs[q][tid] = 0.f;
    }
    const size_t vstride = (size_t)g.nv * g.nu;
    const TIn *ys = sino + (size_t)bt * g.nview * vstride;
    for (int v0 = 0; v0 < g.nview; v0 += kViews) {
        const int nvc = min(kViews, g.nview - v0);
        __syncthreads();
        stage_views(sview, views + v0, nvc, tid, 128);
        __syncthreads();
        if (!active) continue;
        for (int vv = 0; vv < nvc; ++vv) {
            const CtView &V = sview[vv];
            const SfCol C = sf_col<CURVED, DD>(V, g, i, j);
            int d0 = (int)floorf(C.T.k0 + 0.5f), d1 = (int)floorf(C.T.k3 + 0.5f);
            // footprint wholly on the detector: its first and last cell edges
            // lie outside the trapezoid
            const bool whole = d0 >= -C.aref && d1 <= g.nu - 1 - C.aref;
            d0 = max(d0, -C.aref);
            d1 = min(d1, g.nu - 1 - C.aref);
            if (d0 > d1) continue;
            const TIn *yv = ys + (size_t)(v0 + vv) * vstride;
            if constexpr (TT) {
                const TtCol T = tt_col(V, g, C, i, j);
                if (d1 - d0 <= 3 && C.sv > 0.f && g.nu >= 4) {
                    // every knot rises with k (slope sv (1 + e) > 0): the
                    // chunk's rows run from the first voxel's lowest knot to
                    // the last voxel's highest
                    int bref0;
                    float frac0;
                    split_cell(fmaf(C.sv, (float)kbeg, C.fv0), bref0, frac0);
                    const float gb = fmaf(C.sv, (float)kbeg, T.g0), ge = fmaf(C.sv, (float)(kend - 1), T.g0);
                    const float relL = fmaf(C.sv, (float)(kend - 1 - kbeg), frac0);
                    const float lo = fminf(fmaf(gb, T.eN, frac0) - T.hN, fmaf(gb, T.eF, frac0) - T.hF);
                    const float hi = fmaxf(fmaf(ge, T.eN, relL) + T.hN, fmaf(ge, T.eF, relL) + T.hF);
                    const int ef = (int)floorf(lo + 0.5f), el = (int)floorf(hi + 0.5f);
                    if (el - ef + 4 <= NR) {
                        float F[4], Fu[4];
                        trap_cells4(C.T, d0, d1, F);
                        const int as = window4(F, C.aref + d0, g.nu, Fu);
                        // Rs[e - ef] = row bref0 + e filtered by Fu, for e in
                        // [ef, el + 3] (zero off the detector)
                        const int va = max(ef, -bref0), vb = min(el, g.nv - 1 - bref0);
                        const TIn *ya = yv + as;
                        for (int e = ef; e < min(va, el + 1); ++e) Rs[e - ef][tid] = 0.f;
#pragma unroll 4
                        for (int e = va; e <= vb; ++e) {
                            const TIn *row = ya + (size_t)(bref0 + e) * g.nu;
                            float R = Fu[0] * ld(row, 0);
                            R = fmaf(Fu[1], ld(row, 1), R);
                            R = fmaf(Fu[2], ld(row, 2), R);
                            R = fmaf(Fu[3], ld(row, 3), R);
                            Rs[e - ef][tid] = R;
                        }
                        for (int e = max(vb + 1, ef); e <= el + 3; ++e) Rs[e - ef][tid] = 0.f;
#pragma unroll 1
                        for (int kk = 0; kk < ZT; ++kk) {
                            if (kbeg + kk >= kend) break;
                            int e0;
                            float Fv[4];
                            tt_rows(C, T, (float)(kbeg + kk), fmaf(C.sv, (float)kk, frac0), e0, Fv);
                            const int ix = min(max(e0 - ef, 0), NR - 4);
                            float s = Fv[0] * Rs[ix][tid];
                            s = fmaf(Fv[1], Rs[ix + 1][tid], s);
                            s = fmaf(Fv[2], Rs[ix + 2][tid], s);
                            s = fmaf(Fv[3], Rs[ix + 3][tid], s);
                            Gs[kk][tid] += s;
                        }
                        continue;
                    }
                }
                // general footprints: each voxel's rows read directly
                for (int db = d0; db <= d1; db += 4) {
                    float Fu[4];
                    trap_cells4(C.T, db, d1, Fu);
                    const int abase = C.aref + db;
                    const int na = min(4, d1 - db + 1);
#pragma unroll 1
                    for (int kk = 0; kk < ZT; ++kk) {
                        const int k = kbeg + kk;
                        if (k >= kend) break;
                        int bref, e0;
                        float vf, Fv[4];
                        split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                        tt_rows(C, T, (float)k, vf, e0, Fv);
                        float s = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int b = bref + e0 + q;
                            if (b < 0 || b >= g.nv) continue;
                            const TIn *row = yv + (size_t)b * g.nu + abase;
                            float r = Fu[0] * ld(row, 0);
                            if (na > 1) r = fmaf(Fu[1], ld(row, 1), r);
                            if (na > 2) r = fmaf(Fu[2], ld(row, 2), r);
                            if (na > 3) r = fmaf(Fu[3], ld(row, 3), r);
                            s = fmaf(Fv[q], r, s);
                        }
                        Gs[kk][tid] += s;
                    }
                }
                continue;
            }
            float rw = 0.f;
            if (RECON) {
                const float fi = (float)i, fj = (float)j;
                const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, V.au[3]));
                const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, V.an[3]));
                const float den2 = CURVED ? fmaf(cu, cu, cn * cn) : cn * cn;
                const float area = 0.5f * ((C.T.k3 - C.T.k0) + (C.T.k2 - C.T.k1));
                rw = V.rc_w / (den2 * area * (2.f * C.hv));
            }
            if (d1 - d0 <= 3 && C.hv < 0.5f && C.sv > 0.f && g.nu >= 4) {
                float F[4], Fu[4];
                if (whole)
                    nc_cells<4>(C.T, d0, d1, F);  // antiderivative at the interior cell edges only
                else
                    trap_cells4(C.T, d0, d1, F);
                int as;
                if (C.aref + d0 <= g.nu - 4) {  // the 4-cell window starts at the footprint
                    as = C.aref + d0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) Fu[q] = F[q];
                } else {
                    as = window4(F, C.aref + d0, g.nu, Fu);
                }
                // Rows relative to the chunk's first voxel: voxel kk sits at
                // rel = frac0 + sv kk rows from row bref0 (0 < sv < 1), so it
                // touches rows e0, e0 + 1 with e0 in [-1, ZT - 1].
                int bref0;
                float frac0;
                split_cell(fmaf(C.sv, (float)kbeg, C.fv0), bref0, frac0);
                const float last = fmaf(C.sv, (float)(kend - 1 - kbeg), frac0);
                const int ef = (int)floorf(frac0 - C.hv + 0.5f), el = (int)floorf(last + C.hv + 0.5f);
                const int va = max(ef, -bref0), vb = min(el, g.nv - 1 - bref0);  // rows on the detector
                const TIn *ya = yv + as;
                for (int e = ef; e < min(va, el + 1); ++e) Rs[e + 1][tid] = 0.f;  // a chunk below the detector zeroes [ef, el] only
                // two rows per step in packed FP32x2 arithmetic (each lane
                // rounds as the scalar form would)
                float2 Fu2[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) Fu2[q] = make_float2(Fu[q], Fu[q]);
                int e = va;
#pragma unroll 2
                for (; e < vb; e += 2) {
                    const TIn *r0 = ya + (size_t)(bref0 + e) * g.nu, *r1 = r0 + g.nu;
                    float2 R = __fmul2_rn(Fu2[0], make_float2(ld(r0, 0), ld(r1, 0)));
                    R = __ffma2_rn(Fu2[1], make_float2(ld(r0, 1), ld(r1, 1)), R);
                    R = __ffma2_rn(Fu2[2], make_float2(ld(r0, 2), ld(r1, 2)), R);
                    R = __ffma2_rn(Fu2[3], make_float2(ld(r0, 3), ld(r1, 3)), R);
                    Rs[e + 1][tid] = R.x;
                    Rs[e + 2][tid] = R.y;
                }
                if (e == vb) {
                    const TIn *row = ya + (size_t)(bref0 + e) * g.nu;
                    float R = Fu[0] * ld(row, 0);
                    R = fmaf(Fu[1], ld(row, 1), R);
                    R = fmaf(Fu[2], ld(row, 2), R);
                    R = fmaf(Fu[3], ld(row, 3), R);
                    Rs[e + 1][tid] = R;
                }
                for (int e = max(vb + 1, ef); e <= el + 1; ++e) Rs[e + 1][tid] = 0.f;
                // axial sweep: the voxels' rectangles [rel - hv, rel + hv]
                // (rel = frac0 + sv kk) abut (sv = 2 hv < 1), so each voxel
                // either lies in the current row e or crosses its upper edge
                // once; d is the distance from its lower edge to that edge.
                const float w = C.sv;
                const float lo0 = frac0 - C.hv;
                const int e0 = lo0 < -0.5f ? -1 : 0;  // == ef
                float d = ((float)e0 + 0.5f) - lo0;
                const float *rp = &Rs[e0 + 1][tid];
                const float wz0 = fmaf((float)kbeg, g.dz, V.o[2]);
                auto step = [&]() {  // the current voxel's row integral; advances the sweep
                    const bool cross = d < w;
                    const float f0 = cross ? d : w;
                    const float sum = fmaf(f0, rp[0], (w - f0) * rp[128]);
                    rp += cross ? 128 : 0;
                    d = (cross ? d + 1.f : d) - w;
                    return sum;
                };
                // voxels in pairs: amplitudes and accumulation in packed FP32x2
#pragma unroll
                for (int kk = 0; kk < ZT; kk += 2) {
                    if (kbeg + kk + 1 < kend) {
                        const float s0 = step(), s1 = step();
                        float2 amp;
                        if (RECON) {
                            amp = make_float2(rw, rw);
                        } else if (DD) {
                            amp = make_float2(1.f, 1.f);
                        } else {
                            const float2 wz2 = make_float2(fmaf((float)kk, g.dz, wz0), fmaf((float)(kk + 1), g.dz, wz0));
                            const float2 t = __ffma2_rn(wz2, wz2, make_float2(C.rxy2, C.rxy2));
                            amp = __fmul2_rn(__fmul2_rn(make_float2(C.invm, C.invm), t),
                                             make_float2(rsqrtf(t.x), rsqrtf(t.y)));
                        }
                        const float2 a2 = __ffma2_rn(amp, make_float2(s0, s1), make_float2(acc[kk], acc[kk + 1]));
                        acc[kk] = a2.x;
                        acc[kk + 1] = a2.y;
                    } else if (kbeg + kk < kend) {
                        const float s0 = step();
                        const float wz = fmaf((float)kk, g.dz, wz0);
                        acc[kk] = fmaf(RECON ? rw : fp_amp<DD>(C, wz), s0, acc[kk]);
                    }
                }
                continue;
            }
            for (int db = d0; db <= d1; db += 4) {
                float Fu[4];
                trap_cells4(C.T, db, d1, Fu);
                const int abase = C.aref + db;
                const int na = min(4, d1 - db + 1);
                for (int kk = 0; kk < ZT; ++kk) {
                    const int k = kbeg + kk;
                    if (k >= kend) break;
                    int bref;
                    float vf;
                    split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                    int e0 = (int)floorf(vf - C.hv + 0.5f), e1 = (int)floorf(vf + C.hv + 0.5f);
                    e0 = max(e0, -bref);
                    e1 = min(e1, g.nv - 1 - bref);
                    float s = 0.f;
                    for (int e = e0; e <= e1; ++e) {
                        const float Fv = overlap(vf - C.hv, vf + C.hv, e - 0.5f, e + 0.5f);
                        const TIn *row = yv + (size_t)(bref + e) * g.nu + abase;
                        float r = Fu[0] * ld(row, 0);
                        if (na > 1) r = fmaf(Fu[1], ld(row, 1), r);
                        if (na > 2) r = fmaf(Fu[2], ld(row, 2), r);
                        if (na > 3) r = fmaf(Fu[3], ld(row, 3), r);
                        s = fmaf(Fv, r, s);
                    }
                    const float wz = fmaf((float)k, g.dz, V.o[2]);
                    Gs[kk][tid] = fmaf(RECON ? rw : fp_amp<DD>(C, wz), s, Gs[kk][tid]);
                }
            }
        }
    }
    if (!active) return;
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < kend) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc[kk] + Gs[kk][tid], out_t);
    }
}

template <typename TIn, int ZT>
__global__ void __launch_bounds__(128)
sf_back_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
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
            const SfVox P = sf_vox_nc(V, g, i, j, k);
            int d0 = (int)floorf(P.T.k0 + 0.5f), d1 = (int)floorf(P.T.k3 + 0.5f);
            d0 = max(d0, -P.aref);
            d1 = min(d1, g.nu - 1 - P.aref);
            int e0 = (int)floorf(P.vlo + 0.5f), e1 = (int)floorf(P.vhi + 0.5f);
            e0 = max(e0, -P.bref);
            e1 = min(e1, g.nv - 1 - P.bref);
            float s = 0.f;
            for (int db = d0; db <= d1; db += 4) {
                float Fu[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) Fu[q] = (db + q <= d1) ? trap_cell(P.T, db + q) : 0.f;
                const int na = min(4, d1 - db + 1);
                for (int e = e0; e <= e1; ++e) {
                    const float Fv = overlap(P.vlo, P.vhi, e - 0.5f, e + 0.5f);
                    const TIn *row = yv + (size_t)(P.bref + e) * g.nu + P.aref + db;
                    float r = Fu[0] * ld(row, 0);
                    if (na > 1) r = fmaf(Fu[1], ld(row, 1), r);
                    if (na > 2) r = fmaf(Fu[2], ld(row, 2), r);
                    if (na > 3) r = fmaf(Fu[3], ld(row, 3), r);
                    s = fmaf(Fv, r, s);
                }
            }
            acc[kk] = fmaf(P.amp, s, acc[kk]);
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
// CTA = 32 detector cells x BV = 8 RPT rows of one view, 256 threads.
// Work items are the voxel columns (slab s, lateral l) whose footprint can
// reach the tile, taken 256 at a time.  Stage 1: thread = item; it computes
// the column's transaxial weights Fu (<= 4 cells) and walks the column down
// z, accumulating its axial projection Z(item, b) = sum_k amp Fv x onto the
// tile's rows in shared memory.  Stage 2: thread = (cell a, RPT rows); it
// finds, per slab of the round, the items that reach its cell and adds
// Fu(item, a) Z(item, b).  Each sum has a fixed order: deterministic, and
// no atomics.  Used when every footprint spans at most 4 cells (decided on
// the host from the per-view footprint bound); otherwise sf_fwd_circ_wide.
constexpr int kItems = 256;
constexpr int kSlabSeg = 256;

template <int RPT, int NA> struct SfFwdSmem {
    float Z[8 * RPT][kItems];  // [row][item]
    // the item's NA transaxial cell weights; rows padded by 8 so that lanes
    // reading one item's weights of different cells fall on different banks
    float Fu[NA][kItems + 8];
    int a0[kItems];
    int L0[kSlabSeg], cnt[kSlabSeg], off[kSlabSeg + 1];
};

// Voxel-driven stage 1 of the streaming forward: the column's centre splits
// between cells floor(fu), floor(fu) + 1 with hat weights, and each voxel's
// centre between rows floor(fv), floor(fv) + 1; Z accumulates amp x hat x.
template <typename TIn, bool CURVED, int BV, int NA>
__device__ __forceinline__ void vx_stage1(const CtView &V, const CtGrid &g, int i, int j, int B0, int bt,
                                          const TIn *__restrict__ x, const TIn *__restrict__ volZ,
                                          float (&Z)[BV][kItems], float (&Fu)[NA][kItems + 8], int *a0, int tid) {
    const VxCol C = vx_col<CURVED>(V, g, i, j);
    const float af = floorf(C.fu), ta = C.fu - af;
    Fu[0][tid] = 1.f - ta;
    Fu[1][tid] = ta;
#pragma unroll
    for (int r = 2; r < NA; ++r) Fu[r][tid] = 0.f;
    a0[tid] = (int)af;
#pragma unroll
    for (int r = 0; r < BV; ++r) Z[r][tid] = 0.f;
    // voxels whose centre projects within one row of the tile
    const float hw = 1.f + kSearchPad;
    const float rsv = 1.f / C.sv;
    const float ka = ((float)B0 - C.fv0 - hw) * rsv;
    const float kb = ((float)(B0 + BV - 1) - C.fv0 + hw) * rsv;
    const int k0 = max(0, (int)ceilf(fminf(ka, kb)));
    const int k1 = min(g.nz - 1, (int)floorf(fmaxf(ka, kb)));
    auto tap = [&](int k, float xv) {
        const float fv = fmaf(C.sv, (float)k, C.fv0);
        const float bf = floorf(fv), tb = fv - bf;
        const float val = vx_amp_col(C, g, V, k) * xv;
        const int r0 = (int)bf - B0;
        if (r0 >= 0 && r0 < BV) Z[r0][tid] = fmaf(1.f - tb, val, Z[r0][tid]);
        if (r0 + 1 >= 0 && r0 + 1 < BV) Z[r0 + 1][tid] = fmaf(tb, val, Z[r0 + 1][tid]);
    };
    if (volZ != nullptr) {  // contiguous column of the z-major copy, 4 voxels per load
        const TIn *cz = volZ + (size_t)bt * g.nx * g.ny * g.nz + ((size_t)j * g.nx + i) * g.nz;
        for (int kq = k0 & ~3; kq <= k1; kq += 4) {
            float xv[4];
            ld4(cz + kq, xv);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (kq + t >= k0 && kq + t <= k1) tap(kq + t, xv[t]);
        }
    } else {
        const TIn *xc = x + (size_t)j * g.nx + i;
        const size_t zs = (size_t)g.nx * g.ny;
#pragma unroll 4
        for (int k = k0; k <= k1; ++k) tap(k, ld(xc, (size_t)k * zs));
    }
}

// SF-TT stage 1 of the streaming forward (flat detector): the column's
// SF-TR transaxial weights are in Fu already; each voxel spreads x over the
// rows of its axial trapezoid (amplitude 1: A2 is applied per cell).
template <typename TIn, int BV>
__device__ __forceinline__ void tt_stage1(const CtView &V, const CtGrid &g, const SfCol &C, int i, int j, int B0,
                                          int bt, const TIn *__restrict__ x, const TIn *__restrict__ volZ,
                                          float (&Z)[BV][kItems], int tid) {
    const TtCol T = tt_col(V, g, C, i, j);
    // voxels with a knot within a row of the tile (knots lie within the
    // view's bound m_tt_v of the centre's projection)
    const float hw = 0.5f + V.m_tt_v + kSearchPad;
    const float rsv = 1.f / C.sv;
    const float ka = ((float)B0 - C.fv0 - hw) * rsv;
    const float kb = ((float)(B0 + BV - 1) - C.fv0 + hw) * rsv;
    const int k0 = max(0, (int)ceilf(fminf(ka, kb)));
    const int k1 = min(g.nz - 1, (int)floorf(fmaxf(ka, kb)));
    auto tap = [&](int k, float xv) {
        int bref, e0;
        float vf, Fv[4];
        split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
        tt_rows(C, T, (float)k, vf, e0, Fv);
        const int r0 = bref + e0 - B0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (r0 + q >= 0 && r0 + q < BV) Z[r0 + q][tid] = fmaf(Fv[q], xv, Z[r0 + q][tid]);
    };
    if (volZ != nullptr) {  // contiguous column of the z-major copy, 4 voxels per load
        const TIn *cz = volZ + (size_t)bt * g.nx * g.ny * g.nz + ((size_t)j * g.nx + i) * g.nz;
#pragma unroll 1
        for (int kq = k0 & ~3; kq <= k1; kq += 4) {
            float xv[4];
            ld4(cz + kq, xv);
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (kq + t >= k0 && kq + t <= k1) tap(kq + t, xv[t]);
        }
    } else {
        const TIn *xc = x + (size_t)j * g.nx + i;
        const size_t zs = (size_t)g.nx * g.ny;
#pragma unroll 1
        for (int k = k0; k <= k1; ++k) tap(k, ld(xc, (size_t)k * zs));
    }
}

// Axial sweep of one column in circular geometry (SF-TR or DD, axial
// rectangle narrower than a row).  Voxel k covers rows [p_k - hv, p_k + hv]
// with p_k = sv k + fv0 and sv = 2 hv, so consecutive rectangles abut: the
// column's axial profile is a step function (value amp x on each voxel's
// rectangle) and Z(row) is its integral over the row.  Walking k upward, a
// voxel either lies inside the current row (adds w val, w = sv) or crosses
// its upper edge once: the part below closes the row, whose sum is stored
// once, and the rest opens the next.  d is the distance from the voxel's
// lower edge to that row edge.  The walk runs over whole groups of four
// voxels from k0 & ~3 (k0 & ~7 when nz is a multiple of 8) to k1 | 3 of the
// z-major column (nz a multiple of 4); voxels outside [k0, k1] reach only
// rows outside the tile, whose sums are dropped.  Rows the walk does not
// reach are zero.
template <typename TIn, bool DD, int BV>
__device__ __forceinline__ void sf_sweep(const SfCol &C, const CtGrid &g, const CtView &V,
                                         const TIn *__restrict__ cz, int k0, int k1, int B0,
                                         float (&Z)[BV][kItems], int tid) {
    // groups of eight from a sector boundary when nz is a multiple of 8
    const int ks = (g.nz & 7) ? (k0 & ~3) : (k0 & ~7), ke = k1 | 3;
    const float w = C.sv;
    int bref;
    float frac;
    split_cell(fmaf(C.sv, (float)ks, C.fv0), bref, frac);
    const float lo = frac - C.hv;  // lower edge, rows from bref: [-1, 0.5)
    const int e0 = lo < -0.5f ? -1 : 0;
    int r = bref + e0 - B0;          // tile row holding the lower edge
    float d = ((float)e0 + 0.5f) - lo;  // to that row's upper edge: (0, 1]
    const int rfirst = r;
    float acc = 0.f;
    const float wz0 = fmaf((float)ks, g.dz, V.o[2]);
    // amplitude x value of voxels ks + t, ks + t + 1, in packed FP32x2
    auto vals = [&](int t, float x0, float x1) {
        if (DD) return make_float2(x0, x1);
        const float2 wz2 = make_float2(fmaf((float)t, g.dz, wz0), fmaf((float)(t + 1), g.dz, wz0));
        const float2 q = __ffma2_rn(wz2, wz2, make_float2(C.rxy2, C.rxy2));
        const float2 amp = __fmul2_rn(__fmul2_rn(make_float2(C.invm, C.invm), q), make_float2(rsqrtf(q.x), rsqrtf(q.y)));
        return __fmul2_rn(amp, make_float2(x0, x1));
    };
    auto step = [&](float val) {
        const bool cross = d < w;
        const float sum = fmaf(cross ? d : w, val, acc);
        const float rest = (w - d) * val;
        if (cross && (unsigned)r < (unsigned)BV) Z[r][tid] = sum;
        acc = cross ? rest : sum;
        r += cross ? 1 : 0;
        d = (cross ? d + 1.f : d) - w;
    };
    // eight voxels (one 32-byte sector of FP32) per iteration
    int kq = ks;
    if ((g.nz & 7) == 0) {  // groups start on 8-element boundaries: one vector load each
        for (; kq + 7 <= ke; kq += 8) {
            float x8[8];
            ld8(cz + kq, x8);
#pragma unroll
            for (int t = 0; t < 8; t += 2) {
                const float2 v2 = vals(kq - ks + t, x8[t], x8[t + 1]);
                step(v2.x);
                step(v2.y);
            }
        }
    }
    for (; kq + 7 <= ke; kq += 8) {
        float x8[8];
        ld4(cz + kq, x8);
        ld4(cz + kq + 4, x8 + 4);
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
            const float2 v2 = vals(kq - ks + t, x8[t], x8[t + 1]);
            step(v2.x);
            step(v2.y);
        }
    }
    if (kq <= ke) {
        float xa[4];
        ld4(cz + kq, xa);
#pragma unroll
        for (int t = 0; t < 4; t += 2) {
            const float2 v2 = vals(kq - ks + t, xa[t], xa[t + 1]);
            step(v2.x);
            step(v2.y);
        }
    }
    if ((unsigned)r < (unsigned)BV) Z[r][tid] = acc;
    for (int q = 0; q < min(rfirst, BV); ++q) Z[q][tid] = 0.f;
    for (int q = max(r + 1, 0); q < BV; ++q) Z[q][tid] = 0.f;
}

// (with up to 4 cells per item the SF-TR, DD and voxel-driven kernels fit 80
// registers: 3 blocks per SM)
// TT: SF-TT (flat detector); the per-cell amplitude A2 is applied after the gather.
template <typename TIn, bool CURVED, bool DD, int RPT, int NA, bool VOX = false, bool TT = false>
__global__ void __launch_bounds__(256, (NA <= 4 && !TT) ? 3 : 2)
sf_fwd_circ(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
            const TIn *__restrict__ volZ, void *__restrict__ sino, int out_t, int tiles_u, int tiles_v) {
    constexpr int BV = 8 * RPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SfFwdSmem<RPT, NA> &S = *reinterpret_cast<SfFwdSmem<RPT, NA> *>(smem_raw);
    int bx = blockIdx.x;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int tv = bx % tiles_v; bx /= tiles_v;
    const int v = bx % g.nview;
    const int bt = bx / g.nview;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int A0 = tu * 32, B0 = tv * BV;
    const int a = A0 + threadIdx.x;
    const CtView &V = views[v];
    const int main_y = V.main_y;
    const SlabCoef sc = slab_coef(V, main_y);
    // search half widths: footprint bound + half a cell, or the hat's one cell
    const float mu = VOX ? 1.f + kSearchPad : (DD ? V.m_dd_u : V.m_sf_u) + 0.5f + kSearchPad;
    const float mv = VOX ? 1.f + kSearchPad : (TT ? V.m_tt_v : V.m_sf_v) + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    const float T1 = Det<CURVED>::ratio_at(V, a - mu), T2 = Det<CURVED>::ratio_at(V, a + mu);
    float acc[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) acc[r] = 0.f;

    for (int seg = 0; seg < nslab; seg += kSlabSeg) {
        const int nseg = min(kSlabSeg, nslab - seg);
        // column range of every slab of the segment for the whole tile
        __syncthreads();
        for (int t = tid; t < nseg; t += 256) {
            int L0, L1, K0, K1, c = 0;
            if (slab_search<CURVED>(V, sc, seg + t, A0 - mu, A0 + 31.f + mu, B0 - mv, B0 + BV - 1.f + mv,
                                    nlat, g.nz, L0, L1, K0, K1))
                c = L1 - L0 + 1;
            S.L0[t] = L0;
            S.cnt[t] = c;
        }
        __syncthreads();
        if (tid == 0) {  // exclusive prefix sum (nseg <= 1024, once per segment)
            int o = 0;
            for (int t = 0; t < nseg; ++t) { S.off[t] = o; o += S.cnt[t]; }
            S.off[nseg] = o;
        }
        __syncthreads();
        const int total = S.off[nseg];
        for (int base = 0; base < total; base += kItems) {
            // ---- stage 1: one item (column) per thread
            const int q = base + tid;
            if (q < total) {
                // slab of item q: last t with off[t] <= q.  The warp searches
                // for its first item (every lane reads the same offsets), then
                // each lane steps forward to its own (a slab holds tens of items)
                const int qw = base + (tid & ~31);
                int lo = 0, hi = nseg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (S.off[mid] <= qw) lo = mid; else hi = mid - 1;
                }
                while (lo < nseg - 1 && S.off[lo + 1] <= q) ++lo;
                const int s = seg + lo;
                const int l = S.L0[lo] + (q - S.off[lo]);
                const int i = main_y ? l : s, j = main_y ? s : l;
                const int sl = tid;  // this item's slot in the shared arrays
                if constexpr (VOX) {
                    vx_stage1<TIn, CURVED, BV, NA>(V, g, i, j, B0, bt, x, volZ, S.Z, S.Fu, S.a0, sl);
                } else {
                const SfCol C = sf_col<CURVED, DD>(V, g, i, j);
                int d0 = (int)floorf(C.T.k0 + 0.5f), d1 = (int)floorf(C.T.k3 + 0.5f);
                float Fu[NA];
                trap_cellsN<NA>(C.T, d0, d1, Fu);
#pragma unroll
                for (int r = 0; r < NA; ++r) S.Fu[r][sl] = Fu[r];
                S.a0[sl] = C.aref + d0;
                // voxels whose axial rectangle can meet a row of the tile
                const float hw = 0.5f + (TT ? V.m_tt_v : C.hv) + kSearchPad;
                const float rsv = 1.f / C.sv;
                const float ka = ((float)B0 - C.fv0 - hw) * rsv;
                const float kb = ((float)(B0 + BV - 1) - C.fv0 + hw) * rsv;
                const int k0 = max(0, (int)ceilf(fminf(ka, kb)));
                const int k1 = min(g.nz - 1, (int)floorf(fmaxf(ka, kb)));
                if (!TT && C.hv < 0.5f && C.sv > 0.f && volZ != nullptr && k0 <= k1) {
                    // axial rectangle shorter than a row, column contiguous in
                    // the z-major copy (nz a multiple of 4): one sweep down z
                    const TIn *cz = volZ + (size_t)bt * g.nx * g.ny * g.nz + ((size_t)j * g.nx + i) * g.nz;
                    sf_sweep<TIn, DD, BV>(C, g, V, cz, k0, k1, B0, S.Z, sl);
                } else {
#pragma unroll
                for (int r = 0; r < BV; ++r) S.Z[r][sl] = 0.f;
                if constexpr (TT) {
                    tt_stage1<TIn, BV>(V, g, C, i, j, B0, bt, x, volZ, S.Z, sl);
                } else {
                const TIn *xc = x + (size_t)j * g.nx + i;
                const size_t zs = (size_t)g.nx * g.ny;
                if (C.hv < 0.5f) {
                    // axial rectangle shorter than a row: at most two rows per voxel
#pragma unroll 4
                    for (int k = k0; k <= k1; ++k) {
                        int bref;
                        float vf;
                        split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                        const float wz = fmaf((float)k, g.dz, V.o[2]);
                        const float val = fp_amp<DD>(C, wz) * ld(xc, (size_t)k * zs);
                        int e0;
                        float Fv0, Fv1;
                        two_rows(vf - C.hv, vf + C.hv, e0, Fv0, Fv1);
                        const int r0 = bref + e0 - B0;
                        if (r0 >= 0 && r0 < BV) S.Z[r0][sl] = fmaf(Fv0, val, S.Z[r0][sl]);
                        if (r0 + 1 >= 0 && r0 + 1 < BV) S.Z[r0 + 1][sl] = fmaf(Fv1, val, S.Z[r0 + 1][sl]);
                    }
                } else {
                    for (int k = k0; k <= k1; ++k) {
                        int bref;
                        float vf;
                        split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                        const float wz = fmaf((float)k, g.dz, V.o[2]);
                        const float val = fp_amp<DD>(C, wz) * ld(xc, (size_t)k * zs);
                        const int e0 = (int)floorf(vf - C.hv + 0.5f), e1 = (int)floorf(vf + C.hv + 0.5f);
                        for (int e = e0; e <= e1; ++e) {
                            const int r = bref + e - B0;
                            if (r >= 0 && r < BV)
                                S.Z[r][sl] = fmaf(overlap(vf - C.hv, vf + C.hv, e - 0.5f, e + 0.5f), val, S.Z[r][sl]);
                        }
                    }
                }
                }
                }
                }
            }
            __syncthreads();
            // ---- stage 2: thread = (cell a, rows B0 + threadIdx.y + 8 r)
            if (a < g.nu) {
                const int qend = min(total, base + kItems);
                int lo = 0, hi = nseg - 1;  // first slab with items in [base, qend)
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (S.off[mid] <= base) lo = mid; else hi = mid - 1;
                }
                for (int t = lo; t < nseg && S.off[t] < qend; ++t) {
                    if (S.cnt[t] == 0) continue;
                    const float fs = (float)(seg + t);
                    const float Bu = fmaf(sc.us, fs, sc.u3), Bn = fmaf(sc.ns, fs, sc.n3);
                    const float la = __fdividef(T1 * Bn - Bu, sc.ul - T1 * sc.nl);
                    const float lb = __fdividef(T2 * Bn - Bu, sc.ul - T2 * sc.nl);
                    const int c0 = max((int)ceilf(fminf(la, lb)) - S.L0[t], 0);
                    const int c1 = min((int)floorf(fmaxf(la, lb)) - S.L0[t], S.cnt[t] - 1);
                    for (int c = c0; c <= c1; ++c) {
                        const int item = S.off[t] + c - base;
                        if (item < 0 || item >= kItems) continue;
                        const int sl = item;
                        const int d = a - S.a0[sl];
                        if (d < 0 || d >= NA) continue;
                        const float w = S.Fu[d][sl];
                        if constexpr (RPT % 2 == 0) {  // row pairs in packed FP32x2
                            const float2 w2 = make_float2(w, w);
#pragma unroll
                            for (int r = 0; r < RPT; r += 2) {
                                const float2 p = __ffma2_rn(
                                    w2, make_float2(S.Z[threadIdx.y + 8 * r][sl], S.Z[threadIdx.y + 8 * r + 8][sl]),
                                    make_float2(acc[r], acc[r + 1]));
                                acc[r] = p.x;
                                acc[r + 1] = p.y;
                            }
                        } else {
#pragma unroll
                            for (int r = 0; r < RPT; ++r) acc[r] = fmaf(w, S.Z[threadIdx.y + 8 * r][sl], acc[r]);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
    if (a < g.nu) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int b = B0 + threadIdx.y + 8 * r;
            if (b < g.nv)
                st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a,
                       DD ? acc[r] * dd_len<CURVED>(V, g, a, b) : (TT ? acc[r] * tt_amp(V, g, a, b) : acc[r]),
                       out_t);
        }
    }
}

// Forward for footprints wider than 4 cells: CTA = 32 x 8 cells; per slab
// the CTA computes the contexts of the columns that reach its tile once into
// shared memory; every cell gathers from the columns and voxels reaching it.
struct SfColS {
    Trap T;
    int aref;
    float sv, fv0, hv, invm, rxy2, rsv;
};
constexpr int kCols = 256;

template <typename TIn, bool CURVED, bool DD>
__global__ void __launch_bounds__(256)
sf_fwd_circ_wide(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
                 void *__restrict__ sino, int out_t, int tiles_u) {
    __shared__ SfColS cols[kCols];
    int bx = blockIdx.x;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int v = bx % g.nview;
    const int bt = bx / g.nview;
    const int a = tu * 32 + threadIdx.x;
    const int b = blockIdx.y * 8 + threadIdx.y;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const bool active = a < g.nu && b < g.nv;
    const CtView &V = views[v];
    const int main_y = V.main_y;
    const SlabCoef sc = slab_coef(V, main_y);
    const float mu = (DD ? V.m_dd_u : V.m_sf_u) + 0.5f + kSearchPad, mv = V.m_sf_v + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    const float T1 = Det<CURVED>::ratio_at(V, a - mu), T2 = Det<CURVED>::ratio_at(V, a + mu);
    const float tile_a = (float)(tu * 32), tile_b = (float)(blockIdx.y * 8);
    float acc = 0.f;
    for (int s = 0; s < nslab; ++s) {
        int L0, L1, K0, K1;
        if (!slab_search<CURVED>(V, sc, s, tile_a - mu, tile_a + 31.f + mu, tile_b - mv, tile_b + 7.f + mv,
                                 nlat, g.nz, L0, L1, K0, K1))
            continue;  // uniform over the CTA
        const float fs = (float)s;
        const float Bu = fmaf(sc.us, fs, sc.u3), Bn = fmaf(sc.ns, fs, sc.n3);
        const float la = (T1 * Bn - Bu) / (sc.ul - T1 * sc.nl);
        const float lb = (T2 * Bn - Bu) / (sc.ul - T2 * sc.nl);
        const int ml0 = (int)ceilf(fminf(la, lb)), ml1 = (int)floorf(fmaxf(la, lb));
        for (int cb = L0; cb <= L1; cb += kCols) {
            const int nc = min(kCols, L1 - cb + 1);
            __syncthreads();
            for (int t = tid; t < nc; t += 256) {
                const int l = cb + t;
                const SfCol C = sf_col<CURVED, DD>(V, g, main_y ? l : s, main_y ? s : l);
                SfColS &Q = cols[t];
                Q.T = C.T; Q.aref = C.aref; Q.sv = C.sv; Q.fv0 = C.fv0; Q.hv = C.hv;
                Q.invm = C.invm; Q.rxy2 = C.rxy2; Q.rsv = 1.f / C.sv;
            }
            __syncthreads();
            if (!active) continue;
            const int l0 = max(ml0, cb), l1 = min(ml1, cb + nc - 1);
            for (int l = l0; l <= l1; ++l) {
                const SfColS &C = cols[l - cb];
                const float Fu = trap_cell(C.T, a - C.aref);
                if (Fu == 0.f) continue;
                const int i = main_y ? l : s, j = main_y ? s : l;
                const float hw = 0.5f + C.hv + kSearchPad;
                const float ka = ((float)b - C.fv0 - hw) * C.rsv, kb = ((float)b - C.fv0 + hw) * C.rsv;
                const int k0 = max(K0, (int)ceilf(fminf(ka, kb)));
                const int k1 = min(K1, (int)floorf(fmaxf(ka, kb)));
                for (int k = k0; k <= k1; ++k) {
                    int bref;
                    float vf;
                    split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                    const int e = b - bref;
                    const float Fv = overlap(vf - C.hv, vf + C.hv, e - 0.5f, e + 0.5f);
                    if (Fv == 0.f) continue;
                    const float wz = fmaf((float)k, g.dz, V.o[2]);
                    acc = fmaf(fp_amp<DD>(C, wz) * Fu * Fv,
                               ld(x, ((size_t)k * g.ny + j) * g.nx + i), acc);
                }
            }
        }
    }
    if (active)
        st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a,
           DD ? acc * dd_len<CURVED>(V, g, a, b) : acc, out_t);
}

template <typename TIn>
__global__ void __launch_bounds__(256)
sf_fwd_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
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
    const float mu = V.m_sf_u + 0.5f + kSearchPad, mv = V.m_sf_v + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    float acc = 0.f;
    for (int s = 0; s < nslab; ++s) {
        int l0, l1, k0, k1;
        if (!search_flat(V, sc, s, a - mu, a + mu, b - mv, b + mv, nlat, g.nz, l0, l1, k0, k1)) continue;
        for (int l = l0; l <= l1; ++l) {
            const int i = main_y ? l : s, j = main_y ? s : l;
            for (int k = k0; k <= k1; ++k) {
                const SfVox P = sf_vox_nc(V, g, i, j, k);
                const int e = b - P.bref;
                const float Fv = overlap(P.vlo, P.vhi, e - 0.5f, e + 0.5f);
                if (Fv == 0.f) continue;
                const float Fu = trap_cell(P.T, a - P.aref);
                if (Fu == 0.f) continue;
                acc = fmaf(P.amp * Fu * Fv, ld(x, ((size_t)k * g.ny + j) * g.nx + i), acc);
            }
        }
    }
    st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc, out_t);
}

// ------------------------------------------------------------ DD cell factor
// y'[b][a] = L_c(a, b) y[b][a] for every view: the per-cell path length of
// the DD weight, applied before the back gather (which then has amplitude 1).
template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(256)
dd_prescale(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ y,
            float *__restrict__ yp, int batch) {
    const size_t nview_cells = (size_t)g.nv * g.nu;
    const size_t total = nview_cells * g.nview * batch;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % g.nu);
        const int b = (int)((t / g.nu) % g.nv);
        const int v = (int)((t / nview_cells) % g.nview);
        yp[t] = dd_len<CURVED>(views[v], g, a, b) * ld(y, t);
    }
}

// ------------------------------------------------------------ z-major copy
// xZ[b][j][i][k] = x[b][k][j][i]: each voxel column contiguous, for the
// forward's column walks.  32 x 33 shared-memory tiles over (i, k).
template <typename T>
__global__ void __launch_bounds__(256)
to_zmajor(const T *__restrict__ x, T *__restrict__ xZ, int nx, int ny, int nz) {
    __shared__ T tile[32][33];
    const int tiles_i = (nx + 31) / 32;
    const int i0 = (blockIdx.x % tiles_i) * 32, k0 = (blockIdx.x / tiles_i) * 32;
    const int j = blockIdx.y;
    const size_t nvox = (size_t)nx * ny * nz;
    const T *src = x + blockIdx.z * nvox;
    T *dst = xZ + blockIdx.z * nvox;
    for (int r = threadIdx.y; r < 32; r += 8) {  // rows of k, coalesced along i
        const int k = k0 + r, i = i0 + threadIdx.x;
        if (i < nx && k < nz) tile[r][threadIdx.x] = src[((size_t)k * ny + j) * nx + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {  // rows of i, coalesced along k
        const int i = i0 + r, k = k0 + threadIdx.x;
        if (i < nx && k < nz) dst[((size_t)j * nx + i) * nz + k] = tile[threadIdx.x][r];
    }
}

// ------------------------------------------------------------ launchers
namespace {
// voxels per thread of the circular footprint backs: 16 on a flat detector
// (7 blocks per SM); 32 on a curved one, whose per-(column, view) set-up
// (arc tangents of the corners) costs more and is shared by twice the voxels
// (5 blocks per SM)
constexpr int kZT = 16, kZTcurved = 32;

template <typename TIn, bool CURVED, bool DD, int RPT, int NA, bool VOX = false, bool TT = false>
cudaError_t fp_fwd_stream(const CtGrid &g, const CtView *views, const TIn *src, void *out, int out_t,
                          int batch, cudaStream_t st) {
    const int tiles_u = (g.nu + 31) / 32, tiles_v = (g.nv + 8 * RPT - 1) / (8 * RPT);
    const size_t smem = sizeof(SfFwdSmem<RPT, NA>);
    cudaError_t e = cudaFuncSetAttribute(sf_fwd_circ<TIn, CURVED, DD, RPT, NA, VOX, TT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // a z-major copy of the volume (pooled workspace) makes every column walk
    // a contiguous, vector-loaded read; without it the walks read strided
    TIn *xZ = nullptr;
    if (g.nz % 4 == 0 && g.nz >= 8) {
        const size_t n = (size_t)g.nx * g.ny * g.nz * batch;
        if (workspace_alloc((void **)&xZ, n * sizeof(TIn), st) != cudaSuccess) {
            cudaGetLastError();
            xZ = nullptr;
        } else {
            dim3 tb(32, 8), tg((unsigned)(((g.nx + 31) / 32) * ((g.nz + 31) / 32)), (unsigned)g.ny,
                               (unsigned)batch);
            to_zmajor<TIn><<<tg, tb, 0, st>>>(src, xZ, g.nx, g.ny, g.nz);
        }
    }
    dim3 blk(32, 8), grd((unsigned)((size_t)tiles_u * tiles_v * g.nview * batch));
    sf_fwd_circ<TIn, CURVED, DD, RPT, NA, VOX, TT><<<grd, blk, smem, st>>>(g, views, src, xZ, out, out_t, tiles_u,
                                                                      tiles_v);
    e = cudaGetLastError();
    if (xZ) {
        const cudaError_t ef = workspace_free(xZ, st);
        if (e == cudaSuccess) e = ef;
    }
    return e;
}

// forward, circular geometry
template <typename TIn, bool CURVED, bool DD>
cudaError_t fp_fwd_circ(const CtGrid &g, const CtView *views, const TIn *src, void *out, int out_t,
                        int batch, cudaStream_t st) {
    // every transaxial footprint spans at most 4 cells when its half width
    // (bounded per view on the host) is at most 1.5 cells
    const float mu = DD ? g.max_m_dd_u : g.max_m_sf_u;
    if (mu <= 1.5f) {
        if (g.nv >= 64) return fp_fwd_stream<TIn, CURVED, DD, 8, 4>(g, views, src, out, out_t, batch, st);
        return fp_fwd_stream<TIn, CURVED, DD, 1, 4>(g, views, src, out, out_t, batch, st);
    }
    if (mu <= 3.5f) {  // up to 8 cells
        if (g.nv >= 64) return fp_fwd_stream<TIn, CURVED, DD, 8, 8>(g, views, src, out, out_t, batch, st);
        return fp_fwd_stream<TIn, CURVED, DD, 1, 8>(g, views, src, out, out_t, batch, st);
    }
    const int tiles_u = (g.nu + 31) / 32;
    dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
    sf_fwd_circ_wide<TIn, CURVED, DD><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
    return cudaGetLastError();
}

template <typename TIn, bool CURVED, bool DD, bool RECON = false, bool TT = false>
cudaError_t fp_back_circ(const CtGrid &g, const CtView *views, const TIn *src, void *out, int out_t,
                         int batch, cudaStream_t st) {
    constexpr int ZT = CURVED ? kZTcurved : kZT;
    const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + ZT - 1) / ZT;
    dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
    sf_back_circ<TIn, CURVED, DD, ZT, RECON, TT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
    return cudaGetLastError();
}

template <typename TIn>
cudaError_t sf_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                        int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    const bool curved = g.variant == GEO_CIRC_CURVED;
    if (dir == 0) {
        if (g.variant == GEO_NONCIRC_FLAT) {
            const int tiles_u = (g.nu + 31) / 32;
            dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
            sf_fwd_nc<TIn><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
            return cudaGetLastError();
        }
        return curved ? fp_fwd_circ<TIn, true, false>(g, views, src, out, out_t, batch, st)
                      : fp_fwd_circ<TIn, false, false>(g, views, src, out, out_t, batch, st);
    }
    if (g.variant == GEO_NONCIRC_FLAT) {
        const int tiles_x = (g.nx + 31) / 32, nzc8 = (g.nz + 7) / 8;
        dim3 blk(32, 4), grd8((unsigned)(tiles_x * nzc8 * batch), (unsigned)((g.ny + 3) / 4));
        sf_back_nc<TIn, 8><<<grd8, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc8);
        return cudaGetLastError();
    }
    return curved ? fp_back_circ<TIn, true, false>(g, views, src, out, out_t, batch, st)
                  : fp_back_circ<TIn, false, false>(g, views, src, out, out_t, batch, st);
}

// DD in circular geometry; the back direction scales the sinogram by L_c
// into a stream-ordered FP32 workspace first
template <typename TIn>
cudaError_t dd_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                        int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    const bool curved = g.variant == GEO_CIRC_CURVED;
    if (dir == 0)
        return curved ? fp_fwd_circ<TIn, true, true>(g, views, src, out, out_t, batch, st)
                      : fp_fwd_circ<TIn, false, true>(g, views, src, out, out_t, batch, st);
    const size_t n = (size_t)g.nview * g.nv * g.nu * batch;
    float *yp = nullptr;
    cudaError_t e = workspace_alloc((void **)&yp, n * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152u * 64u);
    if (curved)
        dd_prescale<TIn, true><<<blocks, 256, 0, st>>>(g, views, src, yp, batch);
    else
        dd_prescale<TIn, false><<<blocks, 256, 0, st>>>(g, views, src, yp, batch);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = curved ? fp_back_circ<float, true, true>(g, views, yp, out, out_t, batch, st)
                   : fp_back_circ<float, false, true>(g, views, yp, out, out_t, batch, st);
    const cudaError_t ef = workspace_free(yp, st);
    return e != cudaSuccess ? e : ef;
}

// DD back in non-circular geometry: the same scaling, then the footprint gather
template <typename TIn>
cudaError_t dd_nc_back(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                       cudaStream_t st) {
    const size_t n = (size_t)g.nview * g.nv * g.nu * batch;
    float *yp = nullptr;
    cudaError_t e = workspace_alloc((void **)&yp, n * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152u * 64u);
    dd_prescale<TIn, false><<<blocks, 256, 0, st>>>(g, views, static_cast<const TIn *>(in), yp, batch);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_nc(1, 1, g, views, 0, yp, out_t, out, batch, st);
    const cudaError_t ef = workspace_free(yp, st);
    return e != cudaSuccess ? e : ef;
}
}  // namespace

// DD backprojection into caller-provided scratch of at least
// batch x nview x nv x nu floats (no allocation).  Non-circular footprints
// beyond the footprint kernels' 8 x 4 cells take the general gather, which
// needs no scratch.
cudaError_t launch_dd_back_scratch(const CtGrid &g, const CtView *views, int in_t, const void *in,
                                   int out_t, void *out, int batch, float *scratch, cudaStream_t st) {
    const size_t n = (size_t)g.nview * g.nv * g.nu * batch;
    const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152u * 64u);
    if (g.variant == GEO_NONCIRC_FLAT) {
        if (!nc_footprint_fits(g, 1)) return launch_dd_nc(1, g, views, in_t, in, out_t, out, batch, st);
        switch (in_t) {
        case 0: dd_prescale<float, false><<<blocks, 256, 0, st>>>(g, views, (const float *)in, scratch, batch); break;
        case 1: dd_prescale<__half, false><<<blocks, 256, 0, st>>>(g, views, (const __half *)in, scratch, batch); break;
        default:
            dd_prescale<__nv_bfloat16, false><<<blocks, 256, 0, st>>>(g, views, (const __nv_bfloat16 *)in, scratch,
                                                                     batch);
            break;
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_nc(1, 1, g, views, 0, scratch, out_t, out, batch, st);
    }
    const bool curved = g.variant == GEO_CIRC_CURVED;
    switch (in_t) {
    case 0:
        curved ? dd_prescale<float, true><<<blocks, 256, 0, st>>>(g, views, (const float *)in, scratch, batch)
               : dd_prescale<float, false><<<blocks, 256, 0, st>>>(g, views, (const float *)in, scratch, batch);
        break;
    case 1:
        curved ? dd_prescale<__half, true><<<blocks, 256, 0, st>>>(g, views, (const __half *)in, scratch, batch)
               : dd_prescale<__half, false><<<blocks, 256, 0, st>>>(g, views, (const __half *)in, scratch, batch);
        break;
    default:
        curved ? dd_prescale<__nv_bfloat16, true><<<blocks, 256, 0, st>>>(g, views, (const __nv_bfloat16 *)in,
                                                                          scratch, batch)
               : dd_prescale<__nv_bfloat16, false><<<blocks, 256, 0, st>>>(g, views, (const __nv_bfloat16 *)in,
                                                                           scratch, batch);
        break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return curved ? fp_back_circ<float, true, true>(g, views, scratch, out, out_t, batch, st)
                  : fp_back_circ<float, false, true>(g, views, scratch, out, out_t, batch, st);
}

namespace {
template <typename TIn>
cudaError_t vx_fwd_t(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                     cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    const bool curved = g.variant == GEO_CIRC_CURVED;
    if (g.nv >= 64)
        return curved ? fp_fwd_stream<TIn, true, false, 8, 2, true>(g, views, src, out, out_t, batch, st)
                      : fp_fwd_stream<TIn, false, false, 8, 2, true>(g, views, src, out, out_t, batch, st);
    return curved ? fp_fwd_stream<TIn, true, false, 1, 2, true>(g, views, src, out, out_t, batch, st)
                  : fp_fwd_stream<TIn, false, false, 1, 2, true>(g, views, src, out, out_t, batch, st);
}
}  // namespace

namespace {
template <typename TIn>
cudaError_t recon_fp_t(int dd, const CtGrid &g, const CtView *views, const void *in, void *out, int out_t,
                       int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    const bool curved = g.variant == GEO_CIRC_CURVED;
    if (dd)
        return curved ? fp_back_circ<TIn, true, true, true>(g, views, src, out, out_t, batch, st)
                      : fp_back_circ<TIn, false, true, true>(g, views, src, out, out_t, batch, st);
    return curved ? fp_back_circ<TIn, true, false, true>(g, views, src, out, out_t, batch, st)
                  : fp_back_circ<TIn, false, false, true>(g, views, src, out, out_t, batch, st);
}
}  // namespace

cudaError_t launch_recon_fp(int dd, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                            void *out, int batch, cudaStream_t st) {
    if (g.variant == GEO_NONCIRC_FLAT) return launch_nc_recon(dd, g, views, in_t, in, out_t, out, batch, st);
    switch (in_t) {
    case 0: return recon_fp_t<float>(dd, g, views, in, out, out_t, batch, st);
    case 1: return recon_fp_t<__half>(dd, g, views, in, out, out_t, batch, st);
    default: return recon_fp_t<__nv_bfloat16>(dd, g, views, in, out, out_t, batch, st);
    }
}

cudaError_t zmajor_copy(int elem_bytes, const void *x, void *xZ, int nx, int ny, int nz, int batch,
                        cudaStream_t st) {
    dim3 tb(32, 8), tg((unsigned)(((nx + 31) / 32) * ((nz + 31) / 32)), (unsigned)ny, (unsigned)batch);
    if (elem_bytes == 4)
        to_zmajor<float><<<tg, tb, 0, st>>>(static_cast<const float *>(x), static_cast<float *>(xZ), nx, ny, nz);
    else
        to_zmajor<__half><<<tg, tb, 0, st>>>(static_cast<const __half *>(x), static_cast<__half *>(xZ), nx, ny, nz);
    return cudaGetLastError();
}

cudaError_t launch_vx_fwd_circ(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return vx_fwd_t<float>(g, views, in, out, out_t, batch, st);
    case 1: return vx_fwd_t<__half>(g, views, in, out, out_t, batch, st);
    default: return vx_fwd_t<__nv_bfloat16>(g, views, in, out, out_t, batch, st);
    }
}

namespace {
template <typename TIn>
cudaError_t sftt_circ_fwd_t(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                            cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (g.max_m_sf_u <= 1.5f) {
        if (g.nv >= 64) return fp_fwd_stream<TIn, false, false, 8, 4, false, true>(g, views, src, out, out_t, batch, st);
        return fp_fwd_stream<TIn, false, false, 1, 4, false, true>(g, views, src, out, out_t, batch, st);
    }
    if (g.nv >= 64) return fp_fwd_stream<TIn, false, false, 8, 8, false, true>(g, views, src, out, out_t, batch, st);
    return fp_fwd_stream<TIn, false, false, 1, 8, false, true>(g, views, src, out, out_t, batch, st);
}
}  // namespace

bool sftt_circ_fits(const CtGrid &g) {
    return g.variant == GEO_CIRC_FLAT && !g.is2d && g.max_m_sf_u <= 3.5f && g.max_m_tt_v <= 1.5f;
}

cudaError_t launch_sftt_circ(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                             void *out, int batch, cudaStream_t st) {
    if (dir == 1) return fp_back_circ<float, false, false, false, true>(g, views, static_cast<const float *>(in),
                                                                        out, out_t, batch, st);
    switch (in_t) {
    case 0: return sftt_circ_fwd_t<float>(g, views, in, out, out_t, batch, st);
    case 1: return sftt_circ_fwd_t<__half>(g, views, in, out, out_t, batch, st);
    default: return sftt_circ_fwd_t<__nv_bfloat16>(g, views, in, out, out_t, batch, st);
    }
}

cudaError_t launch_sf(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st) {
    if (g.variant == GEO_NONCIRC_FLAT && nc_footprint_fits(g, 0))
        return launch_nc(0, dir, g, views, in_t, in, out_t, out, batch, st);
    switch (in_t) {
    case 0: return sf_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return sf_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return sf_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

cudaError_t launch_dd(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st) {
    if (g.variant == GEO_NONCIRC_FLAT) {
        if (!nc_footprint_fits(g, 1)) return launch_dd_nc(dir, g, views, in_t, in, out_t, out, batch, st);
        if (dir == 0) return launch_nc(1, 0, g, views, in_t, in, out_t, out, batch, st);
        switch (in_t) {
        case 0: return dd_nc_back<float>(g, views, in, out, out_t, batch, st);
        case 1: return dd_nc_back<__half>(g, views, in, out, out_t, batch, st);
        default: return dd_nc_back<__nv_bfloat16>(g, views, in, out, out_t, batch, st);
        }
    }
    switch (in_t) {
    case 0: return dd_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return dd_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return dd_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
