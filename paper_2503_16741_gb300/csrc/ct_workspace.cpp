// ct_workspace.cpp -- stream-ordered scratch memory for kernels that need a
// buffer beyond their inputs and outputs (the DD backprojector's scaled
// sinogram).  One memory pool per device, created on first use, whose
// release threshold keeps freed blocks for reuse.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "ct_launch.h"

namespace ctp {
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};

cudaError_t pool_for_current(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    *out = g_pools[dev];
    return cudaSuccess;
}
}  // namespace

cudaError_t workspace_alloc(void **p, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    cudaError_t e = pool_for_current(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

cudaError_t workspace_free(void *p, cudaStream_t st) { return p ? cudaFreeAsync(p, st) : cudaSuccess; }

}  // namespace ctp
