// k_sf.cu -- separable-footprint projector SF-TR (Long, Fessler & Balter
// 2010, cited in Sec. 2.3): trapezoid transaxial footprint from the four
// projected column corners, rectangle axial footprint from the projected
// end points, amplitude dx / max(|cos|, |sin|) of the 3D ray to the voxel
// centre.  Forward and back are gather kernels (no atomics) that evaluate the
// same per-voxel weight functions, so they form a matched pair.
#include "ct_device.cuh"
#include "ct_launch.h"

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

template <bool CURVED>
__device__ __forceinline__ SfCol sf_col(const CtView &V, const CtGrid &g, int i, int j) {
    const float fi = (float)i, fj = (float)j;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, V.au[3]));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, V.an[3]));
    SfCol C;
    float fr;
    split_cell(Det<CURVED>::fu(V, cu, cn), C.aref, fr);
    const float hxu = 0.5f * V.au[0], hxn = 0.5f * V.an[0];
    const float hyu = 0.5f * V.au[1], hyn = 0.5f * V.an[1];
    float t0 = fr + Det<CURVED>::dfu(V, cu, cn, -hxu - hyu, -hxn - hyn);
    float t1 = fr + Det<CURVED>::dfu(V, cu, cn, hxu - hyu, hxn - hyn);
    float t2 = fr + Det<CURVED>::dfu(V, cu, cn, -hxu + hyu, -hxn + hyn);
    float t3 = fr + Det<CURVED>::dfu(V, cu, cn, hxu + hyu, hxn + hyn);
    sort4(t0, t1, t2, t3);
    C.T = Trap{t0, t1, t2, t3};
    const float den = Det<CURVED>::den(cu, cn);
    C.sv = V.Kv * V.av[2] / den;
    C.fv0 = fmaf(V.Kv, V.av[3] / den, V.Cv);
    C.hv = 0.5f * fabsf(C.sv);
    const float wx = fmaf(fi, g.dx, V.o[0]), wy = fmaf(fj, g.dy, V.o[1]);
    C.rxy2 = fmaf(wx, wx, wy * wy);
    C.invm = g.dx / fmaxf(fabsf(wx), fabsf(wy));
    return C;
}

__device__ __forceinline__ float sf_amp(const SfCol &C, const CtGrid &g, const CtView &V, int k) {
    const float wz = fmaf((float)k, g.dz, V.o[2]);
    return C.invm * sqrtf(fmaf(wz, wz, C.rxy2));
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
    P.T = Trap{t0, t1, t2, t3};
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
// all views; reads the 1-4 cells x 1-3 rows of each voxel's footprint.
template <typename TIn, bool CURVED, int ZT>
__global__ void __launch_bounds__(128)
sf_back_circ(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
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
        const SfCol C = sf_col<CURVED>(V, g, i, j);
        int d0 = (int)floorf(C.T.k0 + 0.5f), d1 = (int)floorf(C.T.k3 + 0.5f);
        d0 = max(d0, -C.aref);
        d1 = min(d1, g.nu - 1 - C.aref);
        const TIn *yv = ys + (size_t)v * vstride;
        for (int db = d0; db <= d1; db += 4) {
            float Fu[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) Fu[q] = (db + q <= d1) ? trap_cell(C.T, db + q) : 0.f;
            const int abase = C.aref + db;
            const int na = min(4, d1 - db + 1);
#pragma unroll
            for (int kk = 0; kk < ZT; ++kk) {
                const int k = kbeg + kk;
                if (k >= g.nz) break;
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
                acc[kk] = fmaf(sf_amp(C, g, V, k), s, acc[kk]);
            }
        }
    }
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st(vol, base + (size_t)k * g.ny * g.nx, acc[kk], out_t);
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
        if (k < g.nz) st(vol, base + (size_t)k * g.ny * g.nx, acc[kk], out_t);
    }
}

// ------------------------------------------------------------ forward (gather)
// Thread = one detector cell (a, b) of one view; loops over the slabs of
// the view's main axis; in each slab only the voxels whose footprint can
// reach the cell (a window widened by the per-view footprint bound).
template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(256)
sf_fwd_circ(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
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
        if (!slab_search<CURVED>(V, sc, s, a - mu, a + mu, b - mv, b + mv, nlat, g.nz, l0, l1, k0, k1))
            continue;
        for (int l = l0; l <= l1; ++l) {
            const int i = main_y ? l : s, j = main_y ? s : l;
            const SfCol C = sf_col<CURVED>(V, g, i, j);
            const float Fu = trap_cell(C.T, a - C.aref);
            if (Fu == 0.f) continue;
            for (int k = k0; k <= k1; ++k) {
                int bref;
                float vf;
                split_cell(fmaf(C.sv, (float)k, C.fv0), bref, vf);
                const int e = b - bref;
                const float Fv = overlap(vf - C.hv, vf + C.hv, e - 0.5f, e + 0.5f);
                if (Fv == 0.f) continue;
                acc = fmaf(sf_amp(C, g, V, k) * Fu * Fv, ld(x, ((size_t)k * g.ny + j) * g.nx + i), acc);
            }
        }
    }
    st(sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc, out_t);
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
    st(sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc, out_t);
}

// ------------------------------------------------------------ launchers
namespace {
constexpr int kZT = 8;

template <typename TIn>
cudaError_t sf_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                        int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (dir == 0) {
        const int tiles_u = (g.nu + 31) / 32;
        dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
        if (g.variant == GEO_NONCIRC_FLAT)
            sf_fwd_nc<TIn><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
        else if (g.variant == GEO_CIRC_CURVED)
            sf_fwd_circ<TIn, true><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
        else
            sf_fwd_circ<TIn, false><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
    } else {
        const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + kZT - 1) / kZT;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        if (g.variant == GEO_NONCIRC_FLAT)
            sf_back_nc<TIn, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
        else if (g.variant == GEO_CIRC_CURVED)
            sf_back_circ<TIn, true, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
        else
            sf_back_circ<TIn, false, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_sf(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return sf_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return sf_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return sf_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
