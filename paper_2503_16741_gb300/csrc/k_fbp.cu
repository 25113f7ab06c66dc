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
// kernel's odd taps sit in shared memory; a thread computes four outputs two
// cells apart, sharing their samples along a sliding window.
#include <algorithm>

#include "ct_device.cuh"
#include "ct_launch.h"

namespace ctp {

constexpr int kRampThreads = 256;
constexpr int kRampR = 4;  // outputs per thread, two cells apart

// A thread computes the outputs m0, m0 + 2, m0 + 4, m0 + 6: the taps of
// outputs two cells apart share their samples, so stepping through the odd
// taps slides a window of loaded samples along the row (two new loads per
// tap instead of eight).  Each output's sum is formed exactly as in the
// one-output form (same terms, same order: far taps first).
template <typename TIn, bool CURVED>
__global__ void __launch_bounds__(kRampThreads)
ramp_rows(CtGrid g, const CtView *__restrict__ views, const TIn *in, void *out, int out_t) {
    // (in may equal out: a row is read whole into shared memory before it is written)
    extern __shared__ float sm[];
    const int nu = g.nu;
    float *pw = sm + nu;          // pw[-nu .. 2 nu + 2 kRampR) valid, zero outside [0, nu)
    float *hk = sm + 3 * nu + 2 * kRampR;  // hk[j] = h(2 j + 1)
    const int nodd = nu / 2;      // odd offsets 1, 3, .., < nu
    const size_t row = blockIdx.x;
    const int b = (int)(row % g.nv);
    const int v = (int)((row / g.nv) % g.nview);
    const CtView &V = views[v];
    const float D = V.D;
    const float vp = g.is2d ? 0.f : ((float)b - V.Cv) * g.dv;
    const float step = CURVED ? g.du / D : g.du;
    const TIn *src = in + row * nu;
    for (int n = threadIdx.x; n < nu; n += blockDim.x) {
        const float up = ((float)n - V.Cu) * g.du;
        const float w = CURVED ? V.rc_R * cosf(up / D) * D * rsqrtf(fmaf(D, D, vp * vp))
                               : D * rsqrtf(fmaf(D, D, fmaf(up, up, vp * vp)));
        pw[n] = ld(src, (size_t)n) * w;
        pw[n - nu] = 0.f;
        pw[n + nu] = 0.f;
    }
    for (int n = threadIdx.x; n < 2 * kRampR; n += blockDim.x) pw[2 * nu + n] = 0.f;
    constexpr float kInv2Pi2 = 0.05066059182116889f;  // 1 / (2 pi^2)
    for (int j = threadIdx.x; j < nodd; j += blockDim.x) {
        const float k = (float)(2 * j + 1);
        float d;
        if (CURVED) {
            d = sinf(k * step);
        } else {
            d = k * step;
        }
        hk[j] = -kInv2Pi2 / (d * d);
    }
    __syncthreads();
    const int nthr = (nu + 2 * kRampR - 1) / (2 * kRampR) * 2;  // threads that cover the row
    for (int t = threadIdx.x; t < nthr; t += blockDim.x) {
        const int m0 = (t >> 1) * 2 * kRampR + (t & 1);
        float p0x2[kRampR], acc[kRampR], wm[kRampR], wp[kRampR];
        const int k0 = 2 * nodd - 1;  // the farthest odd tap
#pragma unroll
        for (int r = 0; r < kRampR; ++r) {
            p0x2[r] = 2.f * pw[m0 + 2 * r];
            acc[r] = 0.f;
            wm[r] = pw[m0 + 2 * r - k0];
            wp[r] = pw[m0 + 2 * r + k0];
        }
        for (int j = nodd - 1; j >= 0; --j) {  // far taps (the small ones) first
            const float h = hk[j];
#pragma unroll
            for (int r = 0; r < kRampR; ++r) acc[r] = fmaf(h, (wm[r] + wp[r]) - p0x2[r], acc[r]);
            if (j == 0) break;
            const int k = 2 * j - 1;  // the next tap: the window moves two cells inwards
#pragma unroll
            for (int r = 0; r < kRampR - 1; ++r) wm[r] = wm[r + 1];
            wm[kRampR - 1] = pw[m0 + 2 * (kRampR - 1) - k];
#pragma unroll
            for (int r = kRampR - 1; r > 0; --r) wp[r] = wp[r - 1];
            wp[0] = pw[m0 + k];
        }
#pragma unroll
        for (int r = 0; r < kRampR; ++r) {
            const int m = m0 + 2 * r;
            if (m < nu) st(out, row * nu + m, fmaf(step, acc[r], V.rc_c * (0.5f * p0x2[r])), out_t);
        }
    }
}

namespace {
template <typename TIn>
cudaError_t ramp_t(const CtGrid &g, const CtView *views, const void *in, void *out, int out_t, int batch,
                   cudaStream_t s) {
    const size_t smem = sizeof(float) * (3 * (size_t)g.nu + 2 * kRampR + g.nu / 2 + 1);
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
