// ct_launch.h -- internal kernel launchers, one per projector.
// dir: 0 = forward (volume -> sinogram), 1 = back (sinogram -> volume).
// in_t / out_t: 0 f32, 1 f16, 2 bf16.  All launches are asynchronous on st.
#pragma once
#include <cuda_runtime.h>

#include "ct_types.h"

namespace ctp {

cudaError_t launch_sf(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st);
cudaError_t launch_dd(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st);
cudaError_t launch_dd_nc(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                         int out_t, void *out, int batch, cudaStream_t st);
// SF-TR (kind 0), DD (1) or SF-TT (2) with per-voxel footprints (any flat
// detector) of at most 8 cells by 4 rows (nc_footprint_fits); the DD and
// SF-TT back directions take the sinogram already scaled by each cell's
// factor (launch_sftt does that for SF-TT).
bool nc_footprint_fits(const CtGrid &g, int kind);
cudaError_t launch_sftt(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                        void *out, int batch, cudaStream_t st);
// SF-TT in circular flat 3D geometry on the streaming forward and the
// column-walk back (k_sf.cu), for transaxial footprints of at most 8 cells and
// axial ones of at most 4 rows; the back direction takes the FP32 sinogram
// already scaled by the per-cell amplitude (in_t ignored).
bool sftt_circ_fits(const CtGrid &g);
cudaError_t launch_sftt_circ(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                             void *out, int batch, cudaStream_t st);
cudaError_t launch_nc(int kind, int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                      int out_t, void *out, int batch, cudaStream_t st);
// voxel-driven forward in circular geometry (the streaming forward of k_sf.cu)
cudaError_t launch_vx_fwd_circ(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st);
// recon mode (FBP): the pre-weighted ramp filter of each detector row, and the
// depth-weighted voxel-driven backprojection of the filtered projections
cudaError_t launch_ramp_filter(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st);
// recon mode with the normalised DD (dd = 1) or SF-TR (dd = 0) footprints;
// non-circular footprints beyond 8 x 4 give cudaErrorNotSupported
cudaError_t launch_recon_fp(int dd, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                            void *out, int batch, cudaStream_t st);
cudaError_t launch_nc_recon(int dd, const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                            void *out, int batch, cudaStream_t st);
cudaError_t launch_voxel_recon(const CtGrid &g, const CtView *views, int in_t, const void *in, int out_t,
                               void *out, int batch, cudaStream_t st);
cudaError_t launch_voxel(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                         int out_t, void *out, int batch, cudaStream_t st);
cudaError_t launch_ray(int dir, const CtGrid &g, const CtView *views, int in_t, const void *in,
                       int out_t, void *out, int batch, cudaStream_t st);

cudaError_t launch_dd_back_scratch(const CtGrid &g, const CtView *views, int in_t, const void *in,
                                   int out_t, void *out, int batch, float *scratch, cudaStream_t st);

// xZ[b][j][i][k] = x[b][k][j][i] for elements of elem_bytes (2 or 4) bytes
cudaError_t zmajor_copy(int elem_bytes, const void *x, void *xZ, int nx, int ny, int nz, int batch,
                        cudaStream_t st);

// Stream-ordered scratch from a library-owned pool on the current device
// (memory is kept in the pool between calls, so steady-state calls do not
// reach the driver's allocator).
cudaError_t workspace_alloc(void **p, size_t bytes, cudaStream_t st);
cudaError_t workspace_free(void *p, cudaStream_t st);
// release threshold of the current device's pool (and a trim to it)
cudaError_t workspace_set_limit(size_t bytes);
// bytes the pool holds from the device now, and the high-water mark of the
// bytes in use (reset to zero when reset_high is set)
cudaError_t workspace_usage(size_t *reserved, size_t *used_high, int reset_high);

}  // namespace ctp
