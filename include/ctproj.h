/*
 * ctproj.h -- C ABI of the GB300 CT projector library (libctproj.so).
 *
 * The library computes the forward projection y = A x and its adjoint
 * backprojection x = A^T y of CTorch (arXiv 2503.16741, Sec. 2.3, Eq. 1 and
 * Eq. 2) for the scan geometries of Sec. 2.2 (2D fan beam, 3D circular and
 * non-circular cone beam, flat or curved detector, per-view parameters) and
 * the four projector algorithms of Sec. 2.3 (voxel-driven, ray-driven,
 * distance-driven, separable footprint).  The system matrix A is never
 * stored; every call recomputes its weights on the GPU (Sec. 2.3).
 *
 * Data layout (Sec. 1, "batched and channeled" PyTorch tensors):
 *   volume   [batch][nz][ny][nx], x fastest   (2D: nz = 1)
 *   sinogram [batch][nview][nv][nu], u fastest (2D: nv = 1)
 * where batch = B * C of the PyTorch tensor.  Buffers are contiguous device
 * memory owned by the caller.
 *
 * Threading: every call is asynchronous on the CUDA stream it is given and
 * performs no host-device synchronisation.  ct_geometry_create /
 * ct_geometry_destroy allocate and free the device copy of the per-view
 * geometry table on the current device.  Some projections take a
 * stream-ordered workspace from a library-owned memory pool on the current
 * device (kept in the pool between calls, so steady-state calls do not reach
 * the driver's allocator) and return it on the same stream:
 *   ct_back with CT_DD or CT_SF_TT, and with CT_RAY in circular geometry:
 *     the sinogram scaled by each cell's path length, amplitude or secant,
 *     batch x nview x nv x nu floats (non-circular CT_DD only when its
 *     footprints fit the footprint kernels, at most 8 cells by 4 rows);
 *   ct_forward with CT_SF or CT_DD (circular geometry with nz a multiple
 *     of 4 and at least 8, or non-circular geometry), with CT_SF_TT, and
 *     with CT_VOXEL (the same circular cases): a z-major copy of the volume,
 *     batch x nz x ny x nx elements of in_t (skipped, at some speed, when it
 *     cannot be had).
 * ct_workspace_bytes gives that size for a call; ct_workspace_limit caps
 * what the pool keeps once calls have returned it.
 * Results are deterministic: no atomics, fixed summation order.
 *
 * Errors: each call returns a ct_status; ct_last_error() gives a message for
 * the last non-OK status returned on the calling thread.
 */
#ifndef CTPROJ_H
#define CTPROJ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scan geometry kinds (Sec. 2.2, Table 1). */
typedef enum {
    CT_FAN2D = 0,      /* 2D fan beam: theta, SAD, SDD, x_src, x/y_ofst, u_ofst      */
    CT_CIRC3D = 1,     /* 3D circular cone beam: adds z_src, z_ofst, v_ofst          */
    CT_NONCIRC3D = 2   /* 3D non-circular: adds phi (about x) and psi (about y)      */
} ct_geom_kind;

/* Detector models (Sec. 2.2): flat panel, or a cylindrical arc centred on the
   source (curved detectors exist for CT_FAN2D and CT_CIRC3D only, Sec. 2.3). */
typedef enum { CT_DET_FLAT = 0, CT_DET_CURVED = 1 } ct_det_kind;

/* Projector algorithms (Sec. 2.3). */
typedef enum {
    CT_VOXEL = 0,  /* voxel-driven: point voxel, bilinear detector interpolation (Peters 1981) */
    CT_RAY = 1,    /* ray-driven: exact chord lengths of the cell-centre ray (Siddon 1985)     */
    CT_DD = 2,     /* distance-driven: boundary overlaps (De Man & Basu 2004)                 */
    CT_SF = 3,     /* separable footprint SF-TR: trapezoid x rectangle (Long et al. 2010)     */
    CT_SF_TT = 4   /* SF-TT: trapezoid x trapezoid, amplitude per detector cell ("A2"; the
                      same paper's variant for large cone angles); flat detectors, square
                      voxels, footprints of at most 8 cells x 4 rows (else UNSUPPORTED)   */
} ct_projector;

/* Projection modes (Sec. 2.3): "proj" is the matched pair; "recon" is the
   backprojection of filtered backprojection (FBP), which carries a
   depth-dependent weighting instead of the projector's own weights (after
   Kak & Slaney 2001): ct_back backprojects ramp-filtered projections
   (ct_ramp_filter), interpolating with the voxel-driven bilinear hat
   (CT_VOXEL) or with the DD / SF-TR footprints normalised to a unit total
   (CT_DD, CT_SF; non-circular footprints of at most 8 cells x 4 rows), and
   weighting each view by
     flat detector:   dbeta R D / ((X - s).n)^2
     curved detector: dbeta / rho^2,  rho = distance of X from the source axis
   where D is the source-detector distance (flat) or detector radius (curved),
   R = (O - s).n the source's distance to the rotation centre O = 0 along the
   detector normal, and dbeta the view's share of the gantry angle (half the
   angular gaps to the nearest distinct view angles on either side;
   2 pi / nview for pose-given geometries).  CT_RAY and CT_SF_TT, and
   ct_forward, return CT_ERR_UNSUPPORTED in recon mode. */
typedef enum { CT_MODE_PROJ = 0, CT_MODE_RECON = 1 } ct_mode;

/* Storage types of volume and sinogram.  Arithmetic is FP32 in all cases;
   half types are converted on load and rounded once on store. */
typedef enum { CT_F32 = 0, CT_F16 = 1, CT_BF16 = 2 } ct_dtype;

typedef enum {
    CT_OK = 0,
    CT_ERR_INVALID_ARG = 1,   /* bad size, pointer, vector length or geometry          */
    CT_ERR_UNSUPPORTED = 2,   /* valid request outside what the library implements     */
    CT_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed           */
    CT_ERR_OOM = 4,           /* device allocation failed                              */
    CT_ERR_TIMEOUT = 5        /* reserved for host-side watchdogs of callers           */
} ct_status;

/* Geometry description (Sec. 2.2 and Table 1).  Lengths in mm, angles in
 * radians.  Each per-view parameter is an array of length n_<name>, which
 * must be 1 (shared by all views) or nview (one value per view); a NULL
 * pointer means 0.0 for every view.  sad and sdd must be given.
 *
 * World frame: origin at the rotation centre; at theta = 0 the y axis is
 * normal to the detector, the source is at (x_src, SAD, z_src) and the
 * detector centre at (-u_ofst, SAD - SDD, -v_ofst), with detector axes
 * e_u = (1,0,0) and e_v = (0,0,1).  The gantry rotation R = Rz(theta)
 * Rx(phi) Ry(psi) (rotation order y, then x, then z) moves source and
 * detector; the object stays fixed.  Voxel (i,j,k) is centred at
 * ((i-(nx-1)/2) dx + x_ofst, (j-(ny-1)/2) dy + y_ofst, (k-(nz-1)/2) dz + z_ofst).
 * Detector cell (a,b) is centred at u = (a-(nu-1)/2) du, v = (b-(nv-1)/2) dv
 * from the detector centre along e_u, e_v; on a curved detector u is the arc
 * length on the cylinder of radius SDD around the axis through the source
 * along e_v.  For CT_FAN2D, nz and nv must be 1 and dz, dv, z_src, z_ofst,
 * v_ofst, phi, psi are ignored.
 *
 * poses (optional, CT_NONCIRC3D only): nview x 12 doubles per view
 * (source xyz, detector-centre xyz, e_u xyz, e_v xyz) replacing the angle
 * parametrisation; e_u and e_v must be orthonormal.  The object offsets still
 * apply.  The volume must lie in front of the source and behind nothing: for
 * every view each volume corner must be between the source and the detector
 * plane (flat) or cylinder (curved), else CT_ERR_INVALID_ARG. */
typedef struct {
    int kind;                  /* ct_geom_kind */
    int det;                   /* ct_det_kind  */
    int nx, ny, nz;
    double dx, dy, dz;
    int nu, nv;
    double du, dv;             /* du is an arc length on a curved detector */
    int nview;
    const double *theta, *phi, *psi;            int n_theta, n_phi, n_psi;
    const double *sad, *sdd;                    int n_sad, n_sdd;
    const double *x_src, *z_src;                int n_x_src, n_z_src;
    const double *x_ofst, *y_ofst, *z_ofst;     int n_x_ofst, n_y_ofst, n_z_ofst;
    const double *u_ofst, *v_ofst;              int n_u_ofst, n_v_ofst;
    const double *poses;
} ct_geometry_desc;

typedef struct ct_geometry ct_geometry;

/* Validate the description, compute the per-view tables in FP64 (source,
 * detector frame, voxel-index-to-detector maps, footprint search margins),
 * round them once to FP32 and upload them to the current CUDA device.
 * The description's arrays are copied; the caller may free them afterwards.
 * On success *out owns the tables until ct_geometry_destroy.
 * Returns CT_ERR_INVALID_ARG for a malformed description,
 * CT_ERR_UNSUPPORTED for a curved non-circular geometry (Sec. 2.3),
 * CT_ERR_OOM / CT_ERR_CUDA for device failures. */
ct_status ct_geometry_create(const ct_geometry_desc *desc, ct_geometry **out);

/* Free the device table and the host copy.  NULL is accepted. */
ct_status ct_geometry_destroy(ct_geometry *geom);

/* Sizes of the geometry: nx, ny, nz, nu, nv, nview (any pointer may be NULL). */
ct_status ct_geometry_shape(const ct_geometry *geom, int *nx, int *ny, int *nz,
                            int *nu, int *nv, int *nview);

/* Forward projection y = A x (Sec. 2.3, Eq. 1).
 * vol:  device pointer, batch x nz x ny x nx elements of type in_t.
 * sino: device pointer, batch x nview x nv x nu elements of type out_t;
 *       overwritten (not accumulated).
 * batch: number of independent volumes (B*C), >= 1.
 * cuda_stream: cudaStream_t to launch on (NULL = the default stream).
 * The projector's weights follow the cited method of Sec. 2.3; the same
 * weight functions serve ct_back, so the pair is matched to FP32 rounding.
 * CT_SF needs dx == dy.  Inputs and outputs must not overlap.
 * Must be called with the geometry's device current. */
ct_status ct_forward(const ct_geometry *geom, ct_projector proj, ct_mode mode,
                     ct_dtype in_t, const void *vol, ct_dtype out_t, void *sino,
                     int batch, void *cuda_stream);

/* Backprojection x = A^T y, the exact adjoint of ct_forward (Sec. 2.3, Eq. 2).
 * sino: device pointer, batch x nview x nv x nu elements of type in_t.
 * vol:  device pointer, batch x nz x ny x nx elements of type out_t;
 *       overwritten.  Other arguments as for ct_forward.
 * CT_DD, CT_SF_TT and CT_RAY in circular geometry (its sinogram scaled by
 * each cell ray's secant against its horizontal path) use the pooled
 * stream-ordered workspace of the threading note above; CT_ERR_OOM when it
 * cannot be had. */
ct_status ct_back(const ct_geometry *geom, ct_projector proj, ct_mode mode,
                  ct_dtype in_t, const void *sino, ct_dtype out_t, void *vol,
                  int batch, void *cuda_stream);

/* Accumulating forms, for iterative reconstruction (Sec. 2.4: the MBIR
 * gradient step x <- x - lr A^T (A x - y) is one ct_forward_acc with
 * alpha = 1, beta = -1 into a copy of y, then one ct_back_acc with
 * alpha = -lr, beta = 1 into x):
 *   ct_forward_acc:  sino = alpha * A vol   + beta * sino
 *   ct_back_acc:     vol  = alpha * A^T sino + beta * vol
 * Each output element is read (when beta != 0) and written once by the
 * thread that computes it, so the update is in place; the old value is read
 * in out_t and the sum rounded once to out_t.  alpha = 1, beta = 0 is
 * ct_forward / ct_back exactly.  Other arguments, ownership and errors as for
 * ct_forward / ct_back; alpha and beta must be finite. */
ct_status ct_forward_acc(const ct_geometry *geom, ct_projector proj, ct_mode mode,
                         ct_dtype in_t, const void *vol, ct_dtype out_t, void *sino,
                         int batch, float alpha, float beta, void *cuda_stream);
ct_status ct_back_acc(const ct_geometry *geom, ct_projector proj, ct_mode mode,
                      ct_dtype in_t, const void *sino, ct_dtype out_t, void *vol,
                      int batch, float alpha, float beta, void *cuda_stream);

/* Distance-driven backprojection (as ct_back with CT_DD, CT_MODE_PROJ) that
 * allocates no device memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc or take memory from a pool
 * -- a service whose device memory is owned and accounted for by another
 * allocator, a plug-in inside a host application that forbids allocation
 * after start-up, or a latency-critical path that must not risk an
 * allocation.  ct_back's DD path needs a scratch copy of the sinogram scaled
 * by each cell's path length; here that scratch is a fixed device array of
 * 16,777,216 floats (64 MiB) compiled into the library, which every GPU that
 * loads the library holds until the process exits.
 *   geom:  any geometry kind (fan-beam, circular, non-circular);
 *   sino, vol, in_t, out_t, batch, cuda_stream: as for ct_back; the caller
 *          owns both buffers, which must be device memory on the geometry's
 *          device (a host pointer is CT_ERR_INVALID_ARG, as in ct_back).
 * Limit: batch x nview x nv x nu <= 16,777,216, else CT_ERR_INVALID_ARG.
 * The first call on a device looks up the array's device address once (with
 * that device current); make that first call before any stream capture.
 * All calls on a device share the one array: calls whose work overlaps on
 * the GPU (on different streams, or from different threads) race and give
 * wrong results -- serialise them.  The array keeps the previous call's
 * contents; nothing in it needs to start at zero, since each call writes
 * every element it reads.  Results equal ct_back with CT_DD bit for bit. */
ct_status ct_back_dd_noalloc(const ct_geometry *geom, ct_dtype in_t, const void *sino,
                             ct_dtype out_t, void *vol, int batch, void *cuda_stream);

/* The ramp filter of filtered backprojection (the "discrete ramp filter" and
 * "recon" mode of Sec. 2.1 and 2.3; the weights after Kak & Slaney 2001):
 * every detector row of every view is pre-weighted and convolved with the
 * discrete band-limited ramp, in the detector's own coordinates (u_p, v_p
 * from the principal point, the foot of the source's perpendicular):
 *   flat:   p D / sqrt(D^2 + u_p^2 + v_p^2), taps h(0) = 1/(8 du^2),
 *           h(k du) = -1/(2 pi^2 k^2 du^2) for odd k, 0 for even k, times du;
 *   curved: p R cos(u_p / D) D / sqrt(D^2 + v_p^2), taps in the angle
 *           g = du / D: h(0) = 1/(8 g^2), h(k g) = -1/(2 pi^2 sin^2(k g)) for
 *           odd k, times g;
 * zero outside the row.  FBP = ct_ramp_filter, then ct_back with CT_VOXEL in
 * CT_MODE_RECON (full scans; no short-scan weighting).
 * sino, out: device pointers, batch x nview x nv x nu elements of in_t and
 *   out_t; out may equal sino (same type) for an in-place filter.
 * Errors: CT_ERR_INVALID_ARG as for ct_back; CT_ERR_UNSUPPORTED when nu >
 *   16384 (one detector row is held in shared memory).  The paper gives the
 *   filter's name only; the form above is Kak & Slaney's. */
ct_status ct_ramp_filter(const ct_geometry *geom, ct_dtype in_t, const void *sino, ct_dtype out_t, void *out,
                         int batch, void *cuda_stream);

/* Pooled workspace (bytes) that one ct_forward (direction 0) or ct_back
 * (direction 1) call with these arguments takes from the library's pool on
 * top of the caller's buffers (see the list at the top of this header; the
 * paper has no counterpart: this is the memory accounting a server needs to
 * admit requests by a device-memory budget).  Host-only; *bytes = 0 when the
 * call takes none.  Errors: CT_ERR_INVALID_ARG for null pointers, unknown
 * enums, a direction other than 0 / 1 or batch < 1. */
ct_status ct_workspace_bytes(const ct_geometry *geom, ct_projector proj, ct_mode mode, int direction,
                             ct_dtype in_t, int batch, size_t *bytes);

/* Caps the bytes the current device's pool keeps once calls have returned
 * their workspace: blocks above `bytes` go back to the device at the next
 * synchronisation, and what the pool already holds above it is released now
 * (blocks in use are not affected).  Default: the pool keeps everything.
 * Errors: CT_ERR_CUDA if the pool cannot be created or set. */
ct_status ct_workspace_limit(size_t bytes);

/* Current device's pool: bytes it holds from the device now (reserved) and
 * the high-water mark of the bytes in use by projection calls since the last
 * reset (used_high); reset_high != 0 resets that mark to zero after reading
 * it.  Either output pointer may be NULL.  Errors: CT_ERR_CUDA. */
ct_status ct_workspace_usage(size_t *reserved, size_t *used_high, int reset_high);

/* Message for the last non-OK status returned on this thread ("" if none). */
const char *ct_last_error(void);

/* Library version string. */
const char *ct_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CTPROJ_H */
