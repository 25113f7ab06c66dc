// ct_workspace.cpp -- stream-ordered scratch memory for kernels that need a
// buffer beyond their inputs and outputs (the scaled FP32 sinograms of the
// DD, SF-TT and circular ray-driven backs, the z-major volume copy of the
// footprint and voxel-driven forwards).  One memory pool per device, created
// on first use, whose release threshold keeps freed blocks for reuse (all of
// them by default; ct_workspace_limit caps what is kept).
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

cudaError_t workspace_set_limit(size_t bytes) {
    cudaMemPool_t pool;
    cudaError_t e = pool_for_current(&pool);
    if (e != cudaSuccess) return e;
    uint64_t keep = bytes;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    // release what is already held above the limit (blocks in use stay)
    return cudaMemPoolTrimTo(pool, bytes);
}

cudaError_t workspace_usage(size_t *reserved, size_t *used_high, int reset_high) {
    cudaMemPool_t pool;
    cudaError_t e = pool_for_current(&pool);
    if (e != cudaSuccess) return e;
    uint64_t r = 0, h = 0;
    if ((e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &r)) != cudaSuccess) return e;
    if ((e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &h)) != cudaSuccess) return e;
    if (reserved) *reserved = (size_t)r;
    if (used_high) *used_high = (size_t)h;
    if (reset_high) {
        uint64_t zero = 0;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    return e;
}

}  // namespace ctp
