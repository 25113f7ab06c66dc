// k_fbp.cu -- the ramp filter of the recon mode (filtered backprojection;
// Sec. 2.3: FBP's backprojection carries a depth-dependent weighting, after
// Kak & Slaney 2001).  Each detector row is pre-weighted and convolved with
// the discrete ramp in the detector's own coordinates (u_p, v_p measured from
// the principal point):
//   flat:   p_w = p D / sqrt(D^2 + u_p^2 + v_p^2), step du,
//           h(0) = 1/(8 du^2), h(k) = -1/(2 pi^2 k^2 du^2) for odd k, 0 for even k
//   curved: p_w = p R cos(u_p / D) D / sqrt(D^2 + v_p^2), step dg = du / D,
//           h(0) = 1/(8 dg^2), h(k) = -1/(2 pi^2 sin^2(k dg)) for odd k
//   q(m) = step sum_n p_w(n) h(m - n)   (zero outside the row)
// The sum is formed as step sum_k h(k) (p_w(m-k) + p_w(m+k) - 2 p_w(m)) +
// rc_c p_w(m), with rc_c = step (h(0) + 2 sum_k h(k)) computed in FP64 on the
// host: the bracket is small where the row is smooth, so FP32 does not lose
// the digits that the large, nearly cancelling taps would cost.
// One CTA per detector row; the row (zero-padded on both sides) and the
// kernel's odd taps sit in shared memory; a thread computes eight outputs two
// cells apart, sharing their samples along a sliding window.
#include <algorithm>

#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

constexpr int kRampThreads = 256;
constexpr int kRampR = 8;  // outputs per thread, two cells apart

// Shared-memory layout of the padded row.  Sample n (zero outside [0, nu))
// sits at logical index n' = n + nu + 48 in [0, 3 nu + 128), stored
// transposed, 16 rows of S: pos(n') = (n' & 15) S + (n' >> 4) with S = 16
// (mod 32).  The lanes of a warp read samples 16 apart (one output group
// each) at two parities; transposed, those fall on 32 distinct banks.
__host__ __device__ constexpr int ramp_off(int nu) { return nu + 48; }
__host__ __device__ constexpr int ramp_len(int nu) { return 3 * nu + 128; }
__host__ __device__ constexpr int ramp_stride(int nu) {
    return ((ramp_len(nu) + 15) / 16 + 15) / 32 * 32 + 16;
}
__device__ __forceinline__ int ramp_pos(int np, int S) { return (np & 15) * S + (np >> 4); }

// A thread computes the outputs m0 + 2 r, r < 8: the taps of outputs two cells
// apart share their samples, so stepping through the odd taps slides a window
// of loaded samples along the row (two new loads per tap instead of sixteen).
// The taps run in groups of eight (the window then turns over once and each
// load's position is a per-lane offset plus a base that moves one column per
// group); taps past the nearest one have h = 0 and leave the sums unchanged.
// Each output's sum is formed exactly as in the one-output form (same terms,
// same order: far taps first).
template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(kRampThreads)
ramp_rows(CtGrid g, const CtView *__restrict__ views, const TIn *in, void *out, int out_t) {
    // (in may equal out: a row is read whole into shared memory before it is written)
    extern __shared__ __align__(16) float sm[];
    constexpr int R = kRampR;
    const int nu = g.nu;
    const int S = ramp_stride(nu), off = ramp_off(nu);
    float *T = sm;                 // the transposed padded row, 16 S floats
    float *hr = sm + 16 * S;       // hr[i] = h(k0 - 2 i), zero for i >= nodd
    const int nodd = nu / 2;       // odd offsets 1, 3, .., < nu
    const int ngrp = (nodd + R - 1) / R;
    const size_t row = blockIdx.x;
    const int b = (int)(row % g.nv);
    const int v = (int)((row / g.nv) % g.nview);
    const CtView &V = views[v];
    const float D = V.D;
    const float vp = g.is2d ? 0.f : ((float)b - V.Cv) * g.dv;
    const float step = CURVED ? g.du / D : g.du;
    const TIn *src = in + row * nu;
    for (int idx = threadIdx.x; idx < 16 * S; idx += blockDim.x) {
        const int n = (idx % S) * 16 + idx / S - off;  // the sample stored at idx
        float val = 0.f;
        if (n >= 0 && n < nu) {
            const float up = ((float)n - V.Cu) * g.du;
            const float w = CURVED ? V.rc_R * cosf(up / D) * D * rsqrtf(fmaf(D, D, vp * vp))
                                   : D * rsqrtf(fmaf(D, D, fmaf(up, up, vp * vp)));
            val = ld(src, (size_t)n) * w;
        }
        T[idx] = val;
    }
    constexpr float kInv2Pi2 = 0.05066059182116889f;  // 1 / (2 pi^2)
    const int k0 = 2 * nodd - 1;  // the farthest odd tap
    for (int i = threadIdx.x; i < ngrp * R; i += blockDim.x) {
        float hv = 0.f;
        if (i < nodd) {
            const float k = (float)(k0 - 2 * i);
            const float d = CURVED ? sinf(k * step) : k * step;
            hv = -kInv2Pi2 / (d * d);
        }
        hr[i] = hv;
    }
    __syncthreads();
    const float4 *hr4 = reinterpret_cast<const float4 *>(hr);
    const int nthr = (nu + 2 * R - 1) / (2 * R) * 2;  // threads that cover the row
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const int m0 = (t >> 1) * 2 * R + (t & 1);
        float p0x2[R], acc[R], wm[R], wp[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            p0x2[r] = 2.f * T[ramp_pos(m0 + 2 * r + off, S)];
            acc[r] = 0.f;
            wm[r] = T[ramp_pos(m0 + 2 * r - k0 + off, S)];
            wp[r] = T[ramp_pos(m0 + 2 * r + k0 + off, S)];
        }
        // the samples loaded after tap i (for tap i + 1): left n' = nL0 + 2 i,
        // right n' = nR0 - 2 i; for i = 8 q + s their positions are
        // (nL0 >> 4) + q + offL[s] and (nR0 >> 4) - q + offR[s]
        const int nL0 = m0 + 2 * (R - 1) - k0 + 2 + off, nR0 = m0 + k0 - 2 + off;
        int offL[R], offR[R];
#pragma unroll
        for (int s = 0; s < R; ++s) {
            offL[s] = ramp_pos(nL0 + 2 * s, S) - (nL0 >> 4);
            offR[s] = ramp_pos(nR0 - 2 * s, S) - (nR0 >> 4);
        }
        int bL = nL0 >> 4, bR = nR0 >> 4;
        for (int q = 0; q < ngrp; ++q, ++bL, --bR) {  // far taps (the small ones) first
            const float4 ha = hr4[2 * q], hb = hr4[2 * q + 1];
            const float h[R] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
            for (int s = 0; s < R; ++s) {
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] = fmaf(h[s], (wm[r] + wp[r]) - p0x2[r], acc[r]);
                // the next tap: the window moves two cells inwards
#pragma unroll
                for (int r = 0; r < R - 1; ++r) wm[r] = wm[r + 1];
                wm[R - 1] = T[bL + offL[s]];
#pragma unroll
                for (int r = R - 1; r > 0; --r) wp[r] = wp[r - 1];
                wp[0] = T[bR + offR[s]];
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int m = m0 + 2 * r;
            if (m < nu) st(out, row * nu + m, fmaf(step, acc[r], V.rc_c * (0.5f * p0x2[r])), out_t);
        }
    }
}

namespace {
template <typename TIn>
cudaError_t ramp_t(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                   cudaStream_t s) {
    const size_t ngrp = ((size_t)g.nu / 2 + kRampR - 1) / kRampR;
    const size_t smem = sizeof(float) * (16 * (size_t)ramp_stride(g.nu) + ngrp * kRampR);
    const TIn *src = static_cast<const TIn *>(in);
    const unsigned rows = (unsigned)((size_t)g.nv * g.nview * batch);
    // as many threads as the row's output groups need (whole warps, 64 .. 256)
    const int groups = (g.nu + 2 * kRampR - 1) / (2 * kRampR) * 2;
    const unsigned threads = (unsigned)std::min(kRampThreads, std::max(64, (groups + 31) / 32 * 32));
    cudaError_t e;
    if (g.variant == GEO_CIRC_CURVED) {
        e = cudaFuncSetAttribute(ramp_rows<TIn, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ramp_rows<TIn, true><<<rows, threads, smem, s>>>(g, views, src, out, out_t);
    } else {
        e = cudaFuncSetAttribute(ramp_rows<TIn, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        ramp_rows<TIn, false><<<rows, threads, smem, s>>>(g, views, src, out, out_t);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_ramp_filter(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st) {
    switch (in_t) {
    case 0: return ramp_t<float>(g, views, in, out, out_t, batch, st);
    case 1: return ramp_t<__half>(g, views, in, out, out_t, batch, st);
    default: return ramp_t<__nv_bfloat16>(g, views, in, out, out_t, batch, st);
    }
}

}  // namespace ctp
