// k_ray.cu -- ray-driven projector (Siddon 1985, cited in Sec. 2.3): the
// weight of voxel j for cell c is the length of the source-to-cell-centre
// segment inside voxel j (half-open voxel boxes).
// Forward: one thread per ray walks the voxel grid from plane crossing to
// plane crossing (parameters measured from the volume entry point).
// Back: the adjoint in gather form -- one thread per voxel column; for each
// view the cells whose central ray can meet the voxel are found from the
// voxel's projected bounding box, and each ray's chord through the voxel is
// computed by the slab method in coordinates centred on the voxel.  In
// circular geometry the x and y slabs of a cell column's rays are shared by
// all its rows and all voxels of the column (ray_back_circ).
#include <algorithm>

#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

// world direction from the source to the centre of cell (a, b)
template <bool CURVED>
__device__ __forceinline__ void ray_dir(const CtView &V, const CtGrid &g, int a, int b, float d[3]) {
    const float Vb = g.dv * ((float)b - V.Cv);
    float cn_, cu_;
    if (CURVED) {
        float sg, cg;
        sincosf(((float)a - V.Cu) / V.Ku, &sg, &cg);
        cn_ = V.D * cg;
        cu_ = V.D * sg;
    } else {
        cn_ = V.D;
        cu_ = g.du * ((float)a - V.Cu);
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) d[m] = fmaf(cn_, V.nn[m], fmaf(cu_, V.eu[m], Vb * V.ev[m]));
}

// ------------------------------------------------------------ forward
template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(256)
ray_fwd(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
        void *__restrict__ sino, int out_t, int tiles_u) {
    int bx = blockIdx.x;
    const int tu = bx % tiles_u; bx /= tiles_u;
    const int v = bx % g.nview;
    const int bt = bx / g.nview;
    const int a = tu * 32 + threadIdx.x;
    const int b = blockIdx.y * 8 + threadIdx.y;
    if (a >= g.nu || b >= g.nv) return;
    const CtView &V = views[v];
    float d[3];
    ray_dir<CURVED>(V, g, a, b, d);
    const float len = sqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
    const float h[3] = {g.dx, g.dy, g.dz};
    const int n[3] = {g.nx, g.ny, g.nz};
    // source and direction in voxel-index units; voxel i spans [i - 1/2, i + 1/2)
    float S[3], D[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        S[m] = -V.o[m] / h[m];
        D[m] = d[m] / h[m];
    }
    float tin = 0.f, tout = 1.f;
    bool hit = true;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float lo = -0.5f, hi = (float)n[m] - 0.5f;
        if (D[m] == 0.f) {
            if (!(S[m] >= lo && S[m] < hi)) hit = false;
        } else {
            const float t1 = (lo - S[m]) / D[m], t2 = (hi - S[m]) / D[m];
            tin = fmaxf(tin, fminf(t1, t2));
            tout = fminf(tout, fmaxf(t1, t2));
        }
    }
    float acc = 0.f;
    if (hit && tout > tin) {
        const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
        // walk from the entry point q; parameters t are measured from it
        float q[3], tn[3], inv[3];
        int cur[3], stp[3];
        const float T = tout - tin;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            q[m] = fmaf(tin, D[m], S[m]);
            if (D[m] > 0.f) {
                cur[m] = (int)floorf(q[m] + 0.5f);
                stp[m] = 1;
            } else if (D[m] < 0.f) {
                cur[m] = (int)ceilf(q[m] - 0.5f);
                stp[m] = -1;
            } else {
                cur[m] = (int)floorf(q[m] + 0.5f);
                stp[m] = 0;
            }
            cur[m] = min(max(cur[m], 0), n[m] - 1);
            inv[m] = D[m] != 0.f ? 1.f / D[m] : 0.f;
            tn[m] = D[m] != 0.f ? ((float)cur[m] + 0.5f * (float)stp[m] - q[m]) * inv[m] : 3.0e38f;
        }
        float tc = 0.f;
        const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
        // every pass steps one axis, so nx + ny + nz + 1 passes cover any ray
        const int max_steps = n[0] + n[1] + n[2] + 1;
        for (int it = 0; it < max_steps && tc < T; ++it) {
            int m = 0;
            float tnext = tn[0];
            if (tn[1] < tnext) { m = 1; tnext = tn[1]; }
            if (tn[2] < tnext) { m = 2; tnext = tn[2]; }
            const float te = fminf(fmaxf(tnext, tc), T);
            acc = fmaf(te - tc, ld(x, (size_t)cur[2] * sz + (size_t)cur[1] * sy + (size_t)cur[0]), acc);
            tc = te;
            cur[m] += stp[m];
            if (cur[m] < 0 || cur[m] >= n[m]) break;
            tn[m] = ((float)cur[m] + 0.5f * (float)stp[m] - q[m]) * inv[m];
        }
        acc *= len;
    }
    st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc, out_t);
}

// ------------------------------------------------------------ back (gather)
// chord of the ray through voxel (centre X, half extents hx, hy, hz) given
// its offset e from the centre (world) and unit direction dh
__device__ __forceinline__ float chord(const float e[3], const float dh[3], const float hh[3]) {
    float lo = -3.0e38f, hi = 3.0e38f;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (dh[m] == 0.f) {
            if (!(e[m] >= -hh[m] && e[m] < hh[m])) return 0.f;
        } else {
            const float inv = 1.f / dh[m];
            const float t1 = (-hh[m] - e[m]) * inv, t2 = (hh[m] - e[m]) * inv;
            lo = fmaxf(lo, fminf(t1, t2));
            hi = fminf(hi, fmaxf(t1, t2));
        }
    }
    return fmaxf(hi - lo, 0.f);
}

// flat detector (the non-circular back): chord of cell (a, b)'s central ray
// through the voxel, from the ray's offset at the voxel's depth cn to the
// voxel centre, formed from the cell-relative positions (a - fu), (b - fv)
__device__ __forceinline__ float ray_weight_flat(const CtView &V, const CtGrid &g, int a, int b, float dfu,
                                                 float dfv, float cn, const float hh[3]) {
    float d[3], e[3];
    ray_dir<false>(V, g, a, b, d);
    const float il = rsqrtf(fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2])));
    const float dh[3] = {d[0] * il, d[1] * il, d[2] * il};
    const float sc = cn / V.D;
    const float eu = sc * g.du * dfu, ev = sc * g.dv * dfv;
#pragma unroll
    for (int m = 0; m < 3; ++m) e[m] = fmaf(eu, V.eu[m], ev * V.ev[m]);
    return chord(e, dh, hh);
}

// ------------------------------------------------------------ back, circular geometry
// With e_v = z and e_u, n horizontal, the ray of cell (a, b) runs along the
// same horizontal line for every row b: per unit of horizontal length lambda
// it moves w_a (horizontal unit direction) and rises sigma = V_b / |d_xy(a)|.
// Measured in lambda from the ray's point at the voxel's depth (offset e from
// the voxel centre), the x and y slabs give an interval T_a that depends on
// the column and the cell column only, the z slab one that depends on
// (k, b) through e_z and sigma; the chord is the length of their overlap
// times sqrt(1 + sigma^2).  That secant depends on the cell only and scales
// the sinogram before the gather (ray_prescale).  Slab tests as in chord():
// half-open boxes, an exactly zero direction component tests the offset.
template <bool CURVED>
__device__ __forceinline__ float ray_sec(const CtView &V, const CtGrid &g, int a, int b) {
    const float Vb = g.dv * ((float)b - V.Cv);
    const float Ua = CURVED ? 0.f : g.du * ((float)a - V.Cu);
    const float h2 = fmaf(Ua, Ua, V.D * V.D);  // |d_xy|^2 (curved: D^2)
    return sqrtf(fmaf(Vb, Vb, h2) / h2);
}

template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(256)
ray_prescale(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ y, float *__restrict__ yp,
             int batch) {
    const size_t nview_cells = (size_t)g.nv * g.nu;
    const size_t total = nview_cells * g.nview * batch;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int a = (int)(t % g.nu);
        const int b = (int)((t / g.nu) % g.nv);
        const int v = (int)((t / nview_cells) % g.nview);
        yp[t] = ray_sec<CURVED>(views[v], g, a, b) * ld(y, t);
    }
}

// one slab of the horizontal path: direction component w, offset e, half width h
__device__ __forceinline__ void slab_xy(float w, float e, float h, float &lo, float &hi, bool &in) {
    if (w == 0.f) {
        if (!(e >= -h && e < h)) in = false;
    } else {
        const float inv = 1.f / w;
        const float t1 = (-h - e) * inv, t2 = (h - e) * inv;
        lo = fmaxf(lo, fminf(t1, t2));
        hi = fminf(hi, fmaxf(t1, t2));
    }
}

// Thread = voxel column over ZT voxels; per view and group of NC cell columns
// the horizontal intervals, then per voxel the rows its box can reach.  The
// column's shadow holds at most 2 cell centres when the footprint bound is
// below one cell (NC = 2, one group), else groups of 4.  The voxel loop is
// not unrolled and its sums sit in shared memory.
template <bool CURVED, int ZT, int NC>
__global__ void __launch_bounds__(128)
ray_back_circ(CtGrid g, const CtView *__restrict__ views, const float *__restrict__ ysec,
              void *__restrict__ vol, int out_t, int tiles_x, int nzc) {
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int kbeg = kc * ZT;
    __shared__ float acc_s[ZT][128];
    const int tid = threadIdx.y * 32 + threadIdx.x;
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc_s[q][tid] = 0.f;
    const float hx = 0.5f * g.dx, hy = 0.5f * g.dy, hz = 0.5f * g.dz;
    const size_t vstride = (size_t)g.nv * g.nu;
    const float *ys = ysec + (size_t)bt * g.nview * vstride;
    const float fi = (float)i, fj = (float)j;
    for (int v = 0; v < g.nview; ++v) {
        const CtView &V = views[v];
        const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, V.au[3]));
        const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, V.an[3]));
        int aref;
        float fr;
        split_cell(Det<CURVED>::fu(V, cu, cn), aref, fr);
        // u extent of the column's shadow: its four corners
        const float hxu = 0.5f * V.au[0], hxn = 0.5f * V.an[0];
        const float hyu = 0.5f * V.au[1], hyn = 0.5f * V.an[1];
        const float t0 = Det<CURVED>::dfu(V, cu, cn, -hxu - hyu, -hxn - hyn);
        const float t1 = Det<CURVED>::dfu(V, cu, cn, hxu - hyu, hxn - hyn);
        const float t2 = Det<CURVED>::dfu(V, cu, cn, -hxu + hyu, -hxn + hyn);
        const float t3 = Det<CURVED>::dfu(V, cu, cn, hxu + hyu, hxn + hyn);
        const float umin = fr + fminf(fminf(t0, t1), fminf(t2, t3));
        const float umax = fr + fmaxf(fmaxf(t0, t1), fmaxf(t2, t3));
        int d0 = (int)ceilf(umin - kSearchPad), d1 = (int)floorf(umax + kSearchPad);
        d0 = max(d0, -aref);
        d1 = min(d1, g.nu - 1 - aref);
        if (d0 > d1) continue;
        // depth range of the column (flat: w.n over the square; curved: rho)
        const float rho = Det<CURVED>::den(cu, cn);
        float dmin, dmax;
        if (CURVED) {
            const float hd = 0.5f * sqrtf(g.dx * g.dx + g.dy * g.dy);
            dmin = rho - hd;
            dmax = rho + hd;
        } else {
            const float hd = fabsf(hxn) + fabsf(hyn);
            dmin = cn - hd;
            dmax = cn + hd;
        }
        const float rdmin = 1.f / dmin, rdmax = 1.f / dmax;
        const float zs = (rho / V.D) * g.dv;  // e_z per row of offset (flat: rho = cn)
        // projected row of voxel k's centre: fv = sv k + fv0 (the depth is the column's)
        const float kd = V.Kv / rho;
        const float sv = kd * V.av[2], fv0 = fmaf(kd, V.av[3], V.Cv);
        const float *yv = ys + (size_t)v * vstride;
        for (int db = d0; db <= d1; db += NC) {
            // per cell column: horizontal interval [lo, hi] (empty past the
            // shadow or when missed), |d_xy| and the curved row term q
            float lo[NC], hi[NC], hr[NC], q[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int d = db + c;
                const int a = aref + d;
                const float dfu = (float)d - fr;
                float wx, wy, ex, ey;
                if (CURVED) {
                    float sg, cg;
                    sincosf(((float)a - V.Cu) / V.Ku, &sg, &cg);
                    wx = fmaf(cg, V.nn[0], sg * V.eu[0]);
                    wy = fmaf(cg, V.nn[1], sg * V.eu[1]);
                    // offset at the foot of the perpendicular from the column centre
                    const float dg = -dfu / V.Ku;
                    const float s2 = sinf(0.5f * dg);
                    const float lat = -rho * sinf(dg);
                    ex = lat * fmaf(cg, V.eu[0], -sg * V.nn[0]);
                    ey = lat * fmaf(cg, V.eu[1], -sg * V.nn[1]);
                    hr[c] = V.D;
                    q[c] = 2.f * s2 * s2;
                } else {
                    const float Ua = g.du * ((float)a - V.Cu);
                    const float hxy = sqrtf(fmaf(Ua, Ua, V.D * V.D));
                    const float rh = 1.f / hxy;
                    wx = fmaf(V.D, V.nn[0], Ua * V.eu[0]) * rh;
                    wy = fmaf(V.D, V.nn[1], Ua * V.eu[1]) * rh;
                    // offset at the column centre's depth
                    const float eo = (cn / V.D) * g.du * dfu;
                    ex = eo * V.eu[0];
                    ey = eo * V.eu[1];
                    hr[c] = hxy;
                    q[c] = 0.f;
                }
                float l = -3.0e38f, h = 3.0e38f;
                bool in = d <= d1;
                slab_xy(wx, ex, hx, l, h, in);
                slab_xy(wy, ey, hy, l, h, in);
                lo[c] = in ? l : 1.f;
                hi[c] = in ? h : 0.f;
            }
            const float *ya = yv + (aref + db);
#pragma unroll 1
            for (int kk = 0; kk < ZT; ++kk) {
                const int k = kbeg + kk;
                if (k >= g.nz) break;
                const float cv = fmaf(V.av[2], (float)k, V.av[3]);
                const float fv = fmaf(sv, (float)k, fv0);
                const float hzv = 0.5f * fabsf(V.av[2]);
                const float c1 = cv - hzv, c2 = cv + hzv;
                const float vmin = fmaf(V.Kv, fminf(c1 * rdmin, c1 * rdmax), V.Cv);
                const float vmax = fmaf(V.Kv, fmaxf(c2 * rdmin, c2 * rdmax), V.Cv);
                const int b0 = max(0, (int)ceilf(vmin - kSearchPad));
                const int b1 = min(g.nv - 1, (int)floorf(vmax + kSearchPad));
                float s = 0.f;
                for (int b = b0; b <= b1; ++b) {
                    const float Vb = g.dv * ((float)b - V.Cv);
                    const float dfv = (float)b - fv;
                    const bool level = Vb == 0.f;  // a horizontal ray: the z slab tests the offset
                    const float rv = level ? 0.f : __frcp_rn(Vb);
                    const float *row = ya + (size_t)b * g.nu;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        const float ez = CURVED ? zs * fmaf(-q[c], (float)b - V.Cv, dfv) : zs * dfv;
                        float l, h;
                        if (level) {
                            const bool inz = ez >= -hz && ez < hz;
                            l = inz ? -3.0e38f : 3.0e38f;
                            h = -l;
                        } else {
                            const float rs = hr[c] * rv;  // 1 / sigma
                            const float z1 = (-hz - ez) * rs, z2 = (hz - ez) * rs;
                            l = fminf(z1, z2);
                            h = fmaxf(z1, z2);
                        }
                        const float w = fminf(hi[c], h) - fmaxf(lo[c], l);
                        if (w > 0.f) s = fmaf(w, row[c], s);
                    }
                }
                acc_s[kk][tid] += s;
            }
        }
    }
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc_s[kk][tid], out_t);
    }
}

// The voxel loop of the non-circular back kernel is not unrolled (its body,
// with the per-cell chord search, appears once in the code, which keeps the
// kernel within the instruction cache); the voxels' sums are kept in shared
// memory.
template <typename TIn, int ZT>
__global__ void __launch_bounds__(128)
ray_back_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
            void *__restrict__ vol, int out_t, int tiles_x, int nzc) {
    int bx = blockIdx.x;
    const int tx = bx % tiles_x; bx /= tiles_x;
    const int kc = bx % nzc;
    const int bt = bx / nzc;
    const int i = tx * 32 + threadIdx.x;
    const int j = blockIdx.y * 4 + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const int kbeg = kc * ZT;
    __shared__ float acc_s[ZT][128];
    const int tid = threadIdx.y * 32 + threadIdx.x;
#pragma unroll
    for (int q = 0; q < ZT; ++q) acc_s[q][tid] = 0.f;
    const float hh[3] = {0.5f * g.dx, 0.5f * g.dy, 0.5f * g.dz};
    const size_t vstride = (size_t)g.nv * g.nu;
    const TIn *ys = sino + (size_t)bt * g.nview * vstride;
    const float fi = (float)i, fj = (float)j;
    for (int v = 0; v < g.nview; ++v) {
        const CtView &V = views[v];
        const TIn *yv = ys + (size_t)v * vstride;
#pragma unroll 1
        for (int kk = 0; kk < ZT; ++kk) {
            const int k = kbeg + kk;
            if (k >= g.nz) break;
            const float fk = (float)k;
            const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, fmaf(V.au[2], fk, V.au[3])));
            const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, fmaf(V.an[2], fk, V.an[3])));
            const float cv = fmaf(V.av[0], fi, fmaf(V.av[1], fj, fmaf(V.av[2], fk, V.av[3])));
            int aref, bref;
            float fr, vr;
            split_cell(fmaf(V.Ku, cu / cn, V.Cu), aref, fr);
            split_cell(fmaf(V.Kv, cv / cn, V.Cv), bref, vr);
            // shadow of the box: its eight corners
            float umin = 3.0e38f, umax = -3.0e38f, vmin = 3.0e38f, vmax = -3.0e38f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float sx = (c & 1) ? 0.5f : -0.5f, sy = (c & 2) ? 0.5f : -0.5f;
                const float sz = (c & 4) ? 0.5f : -0.5f;
                const float du_ = fmaf(sx, V.au[0], fmaf(sy, V.au[1], sz * V.au[2]));
                const float dn_ = fmaf(sx, V.an[0], fmaf(sy, V.an[1], sz * V.an[2]));
                const float dv_ = fmaf(sx, V.av[0], fmaf(sy, V.av[1], sz * V.av[2]));
                const float pu = fmaf(V.Ku, fmaf(du_, cn, -cu * dn_) / ((cn + dn_) * cn), fr);
                const float pv = fmaf(V.Kv, fmaf(dv_, cn, -cv * dn_) / ((cn + dn_) * cn), vr);
                umin = fminf(umin, pu); umax = fmaxf(umax, pu);
                vmin = fminf(vmin, pv); vmax = fmaxf(vmax, pv);
            }
            int d0 = max((int)ceilf(umin - kSearchPad), -aref);
            int d1 = min((int)floorf(umax + kSearchPad), g.nu - 1 - aref);
            int e0 = max((int)ceilf(vmin - kSearchPad), -bref);
            int e1 = min((int)floorf(vmax + kSearchPad), g.nv - 1 - bref);
            float s = 0.f;
            for (int e = e0; e <= e1; ++e) {
                const int b = bref + e;
                const TIn *row = yv + (size_t)b * g.nu;
                for (int d = d0; d <= d1; ++d) {
                    const int a = aref + d;
                    const float w = ray_weight_flat(V, g, a, b, (float)d - fr, (float)e - vr, cn, hh);
                    if (w > 0.f) s = fmaf(w, ld(row, (size_t)a), s);
                }
            }
            acc_s[kk][tid] += s;
        }
    }
    const size_t base = (size_t)bt * g.nz * g.ny * g.nx + (size_t)j * g.nx + i;
#pragma unroll
    for (int kk = 0; kk < ZT; ++kk) {
        const int k = kbeg + kk;
        if (k < g.nz) st_out(g, vol, base + (size_t)k * g.ny * g.nx, acc_s[kk][tid], out_t);
    }
}

// ------------------------------------------------------------ launchers
namespace {
constexpr int kZT = 8;    // voxels per thread, non-circular back
constexpr int kZTc = 16;  // circular back

template <typename TIn>
cudaError_t ray_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                         int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (dir == 0) {
        const int tiles_u = (g.nu + 31) / 32;
        dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
        if (g.variant == GEO_CIRC_CURVED)
            ray_fwd<TIn, true><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
        else
            ray_fwd<TIn, false><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
    } else {
        const int tiles_x = (g.nx + 31) / 32;
        if (g.variant == GEO_NONCIRC_FLAT) {
            const int nzc = (g.nz + kZT - 1) / kZT;
            dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
            ray_back_nc<TIn, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
            return cudaGetLastError();
        }
        // circular: the sinogram times each cell's secant (a stream-ordered
        // FP32 workspace), then the gather
        const size_t n = (size_t)g.nview * g.nv * g.nu * batch;
        float *yp = nullptr;
        cudaError_t e = workspace_alloc((void **)&yp, n * sizeof(float), st);
        if (e != cudaSuccess) return e;
        const unsigned blocks = (unsigned)std::min<size_t>((n + 255) / 256, 152u * 64u);
        const bool curved = g.variant == GEO_CIRC_CURVED;
        if (curved)
            ray_prescale<TIn, true><<<blocks, 256, 0, st>>>(g, views, src, yp, batch);
        else
            ray_prescale<TIn, false><<<blocks, 256, 0, st>>>(g, views, src, yp, batch);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            const int nzc = (g.nz + kZTc - 1) / kZTc;
            dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
            // a shadow narrower than one cell (with the search pad) holds at most 2 cell centres
            const bool two = g.max_m_sf_u < 1.f - 2.f * kSearchPad;
            if (curved && two)
                ray_back_circ<true, kZTc, 2><<<grd, blk, 0, st>>>(g, views, yp, out, out_t, tiles_x, nzc);
            else if (curved)
                ray_back_circ<true, kZTc, 4><<<grd, blk, 0, st>>>(g, views, yp, out, out_t, tiles_x, nzc);
            else if (two)
                ray_back_circ<false, kZTc, 2><<<grd, blk, 0, st>>>(g, views, yp, out, out_t, tiles_x, nzc);
            else
                ray_back_circ<false, kZTc, 4><<<grd, blk, 0, st>>>(g, views, yp, out, out_t, tiles_x, nzc);
            e = cudaGetLastError();
        }
        const cudaError_t ef = workspace_free(yp, st);
        return e != cudaSuccess ? e : ef;
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_ray(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                       int out_t, void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return ray_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return ray_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return ray_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
