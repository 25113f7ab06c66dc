// k_dd.cu -- distance-driven projector (De Man & Basu 2004, cited in Sec.
// 2.3) in non-circular geometry (the circular kernels share the footprint
// kernels of k_sf.cu).  Per view the slabs run along the main axis (x or y, whichever the
// central ray follows more closely).  A voxel's transaxial boundary points
// (+- half a voxel along the other axis) and axial boundary points
// (+- dz/2) are projected to the detector; the weight of cell (a, b) is
// (u overlap / du) (v overlap / dv) L_c, with L_c = slab width / |d_main| the
// path of the cell's central ray through one slab.  Gather kernels for both
// directions, sharing the weight functions.
#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

__device__ __forceinline__ float dd_ratio(float K, float c, float b, float dc, float db) {
    return K * fmaf(dc, b, -c * db) / ((b + db) * b);
}

struct DdVox {
    int aref, bref;
    float ulo, uhi, vlo, vhi;
};

__device__ __forceinline__ DdVox dd_vox_nc(const CtView &V, int i, int j, int k) {
    const float fi = (float)i, fj = (float)j, fk = (float)k;
    const float cu = fmaf(V.au[0], fi, fmaf(V.au[1], fj, fmaf(V.au[2], fk, V.au[3])));
    const float cn = fmaf(V.an[0], fi, fmaf(V.an[1], fj, fmaf(V.an[2], fk, V.an[3])));
    const float cv = fmaf(V.av[0], fi, fmaf(V.av[1], fj, fmaf(V.av[2], fk, V.av[3])));
    DdVox P;
    float fr, vr;
    split_cell(fmaf(V.Ku, cu / cn, V.Cu), P.aref, fr);
    split_cell(fmaf(V.Kv, cv / cn, V.Cv), P.bref, vr);
    const int q = V.main_y ? 0 : 1;
    const float hu = 0.5f * V.au[q], hn = 0.5f * V.an[q];
    const float e1 = fr + dd_ratio(V.Ku, cu, cn, -hu, -hn);
    const float e2 = fr + dd_ratio(V.Ku, cu, cn, hu, hn);
    P.ulo = fminf(e1, e2);
    P.uhi = fmaxf(e1, e2);
    const float hzv = 0.5f * V.av[2], hzn = 0.5f * V.an[2];
    const float f1 = vr + dd_ratio(V.Kv, cv, cn, hzv, hzn);
    const float f2 = vr + dd_ratio(V.Kv, cv, cn, -hzv, -hzn);
    P.vlo = fminf(f1, f2);
    P.vhi = fmaxf(f1, f2);
    return P;
}

// ------------------------------------------------------------ back (gather)
template <typename TIn, int ZT>
__global__ void __launch_bounds__(128)
dd_back_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ sino,
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
            const DdVox P = dd_vox_nc(V, i, j, k);
            int d0 = (int)floorf(P.ulo + 0.5f), d1 = (int)floorf(P.uhi + 0.5f);
            d0 = max(d0, -P.aref);
            d1 = min(d1, g.nu - 1 - P.aref);
            int e0 = (int)floorf(P.vlo + 0.5f), e1 = (int)floorf(P.vhi + 0.5f);
            e0 = max(e0, -P.bref);
            e1 = min(e1, g.nv - 1 - P.bref);
            float s = 0.f;
            for (int e = e0; e <= e1; ++e) {
                const int b = P.bref + e;
                const float Ov = overlap(P.vlo, P.vhi, e - 0.5f, e + 0.5f);
                const TIn *row = yv + (size_t)b * g.nu;
                float r = 0.f;
                for (int d = d0; d <= d1; ++d) {
                    const float Ou = overlap(P.ulo, P.uhi, d - 0.5f, d + 0.5f);
                    r = fmaf(Ou * dd_len<false>(V, g, P.aref + d, b), ld(row, (size_t)(P.aref + d)), r);
                }
                s = fmaf(Ov, r, s);
            }
            acc[kk] += s;
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
template <typename TIn>
__global__ void __launch_bounds__(256)
dd_fwd_nc(CtGrid g, const CtView *__restrict__ views, const TIn *__restrict__ vol,
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
    const float mu = V.m_dd_u + 0.5f + kSearchPad, mv = V.m_sf_v + 0.5f + kSearchPad;
    const int nslab = main_y ? g.ny : g.nx, nlat = main_y ? g.nx : g.ny;
    const TIn *x = vol + (size_t)bt * g.nx * g.ny * g.nz;
    float acc = 0.f;
    for (int s = 0; s < nslab; ++s) {
        int l0, l1, k0, k1;
        if (!search_flat(V, sc, s, a - mu, a + mu, b - mv, b + mv, nlat, g.nz, l0, l1, k0, k1)) continue;
        for (int l = l0; l <= l1; ++l) {
            const int i = main_y ? l : s, j = main_y ? s : l;
            for (int k = k0; k <= k1; ++k) {
                const DdVox P = dd_vox_nc(V, i, j, k);
                const int e = b - P.bref, d = a - P.aref;
                const float Ov = overlap(P.vlo, P.vhi, e - 0.5f, e + 0.5f);
                const float Ou = overlap(P.ulo, P.uhi, d - 0.5f, d + 0.5f);
                if (Ov == 0.f || Ou == 0.f) continue;
                acc = fmaf(Ou * Ov, ld(x, ((size_t)k * g.ny + j) * g.nx + i), acc);
            }
        }
    }
    st_out(g, sino, (((size_t)bt * g.nview + v) * g.nv + b) * g.nu + a, acc * dd_len<false>(V, g, a, b), out_t);
}

// ------------------------------------------------------------ launchers
namespace {
constexpr int kZT = 8;

template <typename TIn>
cudaError_t dd_nc_launch_t(int dir, const CtGrid &g, const CtView *views, const void *in, void *out,
                           int out_t, int batch, cudaStream_t st) {
    const TIn *src = static_cast<const TIn *>(in);
    if (dir == 0) {
        const int tiles_u = (g.nu + 31) / 32;
        dim3 blk(32, 8), grd((unsigned)(tiles_u * g.nview * batch), (unsigned)((g.nv + 7) / 8));
        dd_fwd_nc<TIn><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_u);
    } else {
        const int tiles_x = (g.nx + 31) / 32, nzc = (g.nz + kZT - 1) / kZT;
        dim3 blk(32, 4), grd((unsigned)(tiles_x * nzc * batch), (unsigned)((g.ny + 3) / 4));
        dd_back_nc<TIn, kZT><<<grd, blk, 0, st>>>(g, views, src, out, out_t, tiles_x, nzc);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_dd_nc(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                         int out_t, void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return dd_nc_launch_t<float>(dir, g, views, in, out, out_t, batch, st);
    case 1: return dd_nc_launch_t<__half>(dir, g, views, in, out, out_t, batch, st);
    default: return dd_nc_launch_t<__nv_bfloat16>(dir, g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
