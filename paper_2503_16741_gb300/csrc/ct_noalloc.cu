// ct_noalloc.cu -- a distance-driven backprojection entry point that never
// allocates device memory, for callers that cannot: a service whose device
// memory is owned and budgeted by another allocator, a plug-in running inside
// a host application that forbids allocations after start-up, or code that
// must not risk an allocation (and the implicit synchronisation it may bring)
// on a latency-critical path.  Its scratch -- the sinogram scaled by each
// cell's path length -- lives in a fixed-size device array compiled into the
// library instead of coming from cudaMalloc or a memory pool.  It serves
// every geometry kind: non-circular footprints wider than the footprint
// kernels' 8 cells x 4 rows take the general gather, which needs no scratch.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/ctproj.h"
#include "ct_geometry.h"
#include "ct_launch.h"

namespace {

// 16 Mi floats (64 MiB).  Every GPU that loads the library keeps this array
// until the process exits.
constexpr size_t kScratchFloats = size_t(1) << 24;
static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_addr[kMaxDevices] = {};

ct_status fail(ct_status s, const std::string &m) {
    ctp::set_last_error(m);
    return s;
}

// Device address of the array on the current device, looked up once per
// device (the host-side symbol is only a stand-in, not a device address).
cudaError_t scratch_address(int dev, float **out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ct_status ct_back_dd_noalloc(const ct_geometry *g, ct_dtype in_t, const void *sino, ct_dtype out_t,
                                        void *vol, int batch, void *cuda_stream) {
    if (!g) return fail(CT_ERR_INVALID_ARG, "null geometry");
    if (in_t < CT_F32 || in_t > CT_BF16 || out_t < CT_F32 || out_t > CT_BF16)
        return fail(CT_ERR_INVALID_ARG, "unknown dtype");
    if (!sino || !vol) return fail(CT_ERR_INVALID_ARG, "null data pointer");
    if (batch < 1) return fail(CT_ERR_INVALID_ARG, "batch must be >= 1");
    const size_t need = (size_t)g->nview * g->nv * g->nu * (size_t)batch;
    if (need > kScratchFloats)
        return fail(CT_ERR_INVALID_ARG, "batch x nview x nv x nu = " + std::to_string(need) +
                                            " exceeds the static scratch of " + std::to_string(kScratchFloats) +
                                            " floats");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device)
        return fail(CT_ERR_INVALID_ARG, "the geometry's device is not the current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(CT_ERR_INVALID_ARG, "device index out of range");
    if ((long long)((g->nx + 31) / 32) * ((g->nz + 7) / 8) * batch > 2147483647LL)
        return fail(CT_ERR_INVALID_ARG, "batch too large for one launch");
    // a host or foreign pointer is an argument error, caught before any launch
    ct_status st = ctp::check_device_ptr(sino, "input");
    if (st != CT_OK) return st;
    st = ctp::check_device_ptr(vol, "output");
    if (st != CT_OK) return st;
    float *scratch = nullptr;
    cudaError_t e = scratch_address(dev, &scratch);
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    e = ctp::launch_dd_back_scratch(g->grid, g->dev_views, in_t, sino, out_t, vol, batch, scratch,
                                    static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return fail(CT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return CT_OK;
}
