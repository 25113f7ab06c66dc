"""ctypes binding of libctproj (include/ctproj.h).

Argument marshalling only: shapes, dtypes and pointers are checked here and
every projection runs in the library's CUDA kernels.  The library must have
been built (`paper_2503_16741_gb300.build.build()`); without it every call
raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

CT_OK = 0
STATUS = {0: "CT_OK", 1: "CT_ERR_INVALID_ARG", 2: "CT_ERR_UNSUPPORTED", 3: "CT_ERR_CUDA",
          4: "CT_ERR_OOM", 5: "CT_ERR_TIMEOUT"}
KINDS = {"fan2d": 0, "circ3d": 1, "noncirc3d": 2}
DETS = {"flat": 0, "curved": 1}
PROJECTORS = {"voxel": 0, "ray": 1, "dd": 2, "sf": 3, "sftt": 4}
MODES = {"proj": 0, "recon": 1}
DTYPES = {torch.float32: 0, torch.float16: 1, torch.bfloat16: 2}
PER_VIEW = ("theta", "phi", "psi", "sad", "sdd", "x_src", "z_src",
            "x_ofst", "y_ofst", "z_ofst", "u_ofst", "v_ofst")


class CTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("det", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double),
                ("nview", C.c_int),
                ("theta", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double)),
                ("psi", C.POINTER(C.c_double)),
                ("n_theta", C.c_int), ("n_phi", C.c_int), ("n_psi", C.c_int),
                ("sad", C.POINTER(C.c_double)), ("sdd", C.POINTER(C.c_double)),
                ("n_sad", C.c_int), ("n_sdd", C.c_int),
                ("x_src", C.POINTER(C.c_double)), ("z_src", C.POINTER(C.c_double)),
                ("n_x_src", C.c_int), ("n_z_src", C.c_int),
                ("x_ofst", C.POINTER(C.c_double)), ("y_ofst", C.POINTER(C.c_double)),
                ("z_ofst", C.POINTER(C.c_double)),
                ("n_x_ofst", C.c_int), ("n_y_ofst", C.c_int), ("n_z_ofst", C.c_int),
                ("u_ofst", C.POINTER(C.c_double)), ("v_ofst", C.POINTER(C.c_double)),
                ("n_u_ofst", C.c_int), ("n_v_ofst", C.c_int),
                ("poses", C.POINTER(C.c_double))]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libctproj.so (built in-tree); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2503_16741_gb300.build.build() "
                               "(there is no CPU fallback)")
        lib = C.CDLL(path)
        P = C.POINTER
        lib.ct_geometry_create.argtypes = [P(_Desc), P(C.c_void_p)]
        lib.ct_geometry_destroy.argtypes = [C.c_void_p]
        lib.ct_geometry_shape.argtypes = [C.c_void_p] + [P(C.c_int)] * 6
        sig = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
        lib.ct_forward.argtypes = sig
        lib.ct_back.argtypes = sig
        sig_acc = sig[:-1] + [C.c_float, C.c_float, C.c_void_p]
        lib.ct_forward_acc.argtypes = sig_acc
        lib.ct_back_acc.argtypes = sig_acc
        lib.ct_forward_acc.restype = C.c_int
        lib.ct_back_acc.restype = C.c_int
        lib.ct_back_dd_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                           C.c_int, C.c_void_p]
        lib.ct_back_dd_noalloc.restype = C.c_int
        lib.ct_ramp_filter.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]
        lib.ct_ramp_filter.restype = C.c_int
        lib.ct_workspace_bytes.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                           P(C.c_size_t)]
        lib.ct_workspace_bytes.restype = C.c_int
        lib.ct_workspace_limit.argtypes = [C.c_size_t]
        lib.ct_workspace_limit.restype = C.c_int
        lib.ct_workspace_usage.argtypes = [P(C.c_size_t), P(C.c_size_t), C.c_int]
        lib.ct_workspace_usage.restype = C.c_int
        lib.ct_last_error.restype = C.c_char_p
        lib.ct_version.restype = C.c_char_p
        for f in ("ct_geometry_create", "ct_geometry_destroy", "ct_geometry_shape", "ct_forward", "ct_back"):
            getattr(lib, f).restype = C.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != CT_OK:
        raise CTError(rc, load().ct_last_error().decode())


class Geometry:
    """A scan geometry (Sec. 2.2, Table 1) uploaded to the current CUDA device.

    Keyword arguments follow the paper's parameter names; per-view parameters
    are scalars or length-nview sequences.  `Geometry.from_spec(obj)` reads the
    same attributes from any object that has them."""

    def __init__(self, kind: str, det: str, nx: int, ny: int, nz: int, dx: float, dy: float,
                 dz: float, nu: int, nv: int, du: float, dv: float, nview: int,
                 poses: Optional[np.ndarray] = None, **params):
        lib = load()
        unknown = set(params) - set(PER_VIEW)
        if unknown:
            raise TypeError(f"unknown geometry parameters {sorted(unknown)}")
        if poses is None and ("sad" not in params or "sdd" not in params):
            raise TypeError("sad and sdd are required (unless per-view poses are given)")
        self.kind, self.det = kind, det
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.nu, self.nv, self.nview = int(nu), int(nv), int(nview)
        self.dx, self.dy, self.dz, self.du, self.dv = map(float, (dx, dy, dz, du, dv))
        d = _Desc()
        d.kind, d.det = KINDS[kind], DETS[det]
        d.nx, d.ny, d.nz = self.nx, self.ny, self.nz
        d.dx, d.dy, d.dz = self.dx, self.dy, self.dz
        d.nu, d.nv, d.du, d.dv, d.nview = self.nu, self.nv, self.du, self.dv, self.nview
        self._keep = []
        self._params = {}  # per-view parameters as given (for subset())
        for name in PER_VIEW:  # absent parameters are NULL: 0.0 for every view (sad, sdd: unused with poses)
            if name not in params:
                self._params[name] = np.zeros(1)
                setattr(d, name, C.POINTER(C.c_double)())
                setattr(d, "n_" + name, 0)
                continue
            arr = np.ascontiguousarray(np.atleast_1d(np.asarray(params[name], dtype=np.float64)).ravel())
            self._keep.append(arr)
            self._params[name] = arr
            setattr(d, name, arr.ctypes.data_as(C.POINTER(C.c_double)))
            setattr(d, "n_" + name, int(arr.size))
        self._poses = None
        if poses is not None:
            p = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(self.nview, 12))
            self._keep.append(p)
            self._poses = p
            d.poses = p.ctypes.data_as(C.POINTER(C.c_double))
        else:
            d.poses = C.POINTER(C.c_double)()
        h = C.c_void_p()
        _check(lib.ct_geometry_create(C.byref(d), C.byref(h)))
        self._h = h
        self.device = torch.cuda.current_device()

    @classmethod
    def from_spec(cls, spec) -> "Geometry":
        kw = {n: getattr(spec, n) for n in PER_VIEW}
        return cls(spec.kind, spec.det, spec.nx, spec.ny, spec.nz, spec.dx, spec.dy, spec.dz,
                   spec.nu, spec.nv, spec.du, spec.dv, spec.nview,
                   poses=getattr(spec, "poses", None), **kw)

    def subset(self, views: Sequence[int]) -> "Geometry":
        """The same scan restricted to the listed views, in the listed order
        (an ordered subset, Sec. 2.2: every parameter is per view): its
        projections equal those rows of the full geometry's."""
        views = np.asarray(views, dtype=np.int64).ravel()
        if views.size == 0 or views.min() < 0 or views.max() >= self.nview:
            raise ValueError(f"views must lie in [0, {self.nview})")
        kw = {n: (a if a.size == 1 else a[views]) for n, a in self._params.items()}
        return Geometry(self.kind, self.det, self.nx, self.ny, self.nz, self.dx, self.dy, self.dz,
                        self.nu, self.nv, self.du, self.dv, int(views.size),
                        poses=None if self._poses is None else self._poses[views], **kw)

    @property
    def handle(self) -> C.c_void_p:
        if self._h is None:
            raise RuntimeError("geometry was closed")
        return self._h

    @property
    def is2d(self) -> bool:
        return self.kind == "fan2d"

    @property
    def vol_shape(self):
        return (self.ny, self.nx) if self.is2d else (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.nview, self.nu) if self.is2d else (self.nview, self.nv, self.nu)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ct_geometry_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _batch_of(t: torch.Tensor, inner: Sequence[int], what: str) -> int:
    k = len(inner)
    if tuple(t.shape[-k:]) != tuple(inner):
        raise ValueError(f"{what}: trailing shape {tuple(t.shape[-k:])} != {tuple(inner)}")
    return int(np.prod(t.shape[:-k], dtype=np.int64)) if t.dim() > k else 1


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_tensor(t: torch.Tensor, what: str):
    if not t.is_cuda:
        raise ValueError(f"{what} must be a CUDA tensor (no CPU path)")
    if t.dtype not in DTYPES:
        raise ValueError(f"{what}: dtype {t.dtype} not supported (float32, float16, bfloat16)")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")


def forward_into(geom: Geometry, x: torch.Tensor, y: torch.Tensor, projector: str = "sf",
                 mode: str = "proj", stream=None) -> torch.Tensor:
    """y = A x into a preallocated sinogram tensor (Sec. 2.3, Eq. 1)."""
    _check_tensor(x, "volume")
    _check_tensor(y, "sinogram")
    b = _batch_of(x, geom.vol_shape, "volume")
    if _batch_of(y, geom.sino_shape, "sinogram") != b:
        raise ValueError("volume and sinogram batch sizes differ")
    _check(load().ct_forward(geom.handle, PROJECTORS[projector], MODES[mode], DTYPES[x.dtype],
                             x.data_ptr(), DTYPES[y.dtype], y.data_ptr(), b, _stream_ptr(stream)))
    return y


def back_into(geom: Geometry, y: torch.Tensor, x: torch.Tensor, projector: str = "sf",
              mode: str = "proj", stream=None) -> torch.Tensor:
    """x = A^T y into a preallocated volume tensor (Sec. 2.3, Eq. 2)."""
    _check_tensor(y, "sinogram")
    _check_tensor(x, "volume")
    b = _batch_of(y, geom.sino_shape, "sinogram")
    if _batch_of(x, geom.vol_shape, "volume") != b:
        raise ValueError("volume and sinogram batch sizes differ")
    _check(load().ct_back(geom.handle, PROJECTORS[projector], MODES[mode], DTYPES[y.dtype],
                          y.data_ptr(), DTYPES[x.dtype], x.data_ptr(), b, _stream_ptr(stream)))
    return x


def forward_acc(geom: Geometry, x: torch.Tensor, y: torch.Tensor, alpha: float, beta: float,
                projector: str = "sf", mode: str = "proj", stream=None) -> torch.Tensor:
    """y <- alpha A x + beta y, in place (y's dtype is the storage type)."""
    _check_tensor(x, "volume")
    _check_tensor(y, "sinogram")
    b = _batch_of(x, geom.vol_shape, "volume")
    if _batch_of(y, geom.sino_shape, "sinogram") != b:
        raise ValueError("volume and sinogram batch sizes differ")
    _check(load().ct_forward_acc(geom.handle, PROJECTORS[projector], MODES[mode], DTYPES[x.dtype],
                                 x.data_ptr(), DTYPES[y.dtype], y.data_ptr(), b, float(alpha),
                                 float(beta), _stream_ptr(stream)))
    return y


def back_acc(geom: Geometry, y: torch.Tensor, x: torch.Tensor, alpha: float, beta: float,
             projector: str = "sf", mode: str = "proj", stream=None) -> torch.Tensor:
    """x <- alpha A^T y + beta x, in place."""
    _check_tensor(y, "sinogram")
    _check_tensor(x, "volume")
    b = _batch_of(y, geom.sino_shape, "sinogram")
    if _batch_of(x, geom.vol_shape, "volume") != b:
        raise ValueError("volume and sinogram batch sizes differ")
    _check(load().ct_back_acc(geom.handle, PROJECTORS[projector], MODES[mode], DTYPES[y.dtype],
                              y.data_ptr(), DTYPES[x.dtype], x.data_ptr(), b, float(alpha),
                              float(beta), _stream_ptr(stream)))
    return x


def forward(geom: Geometry, x: torch.Tensor, projector: str = "sf", mode: str = "proj",
            out_dtype: Optional[torch.dtype] = None, stream=None) -> torch.Tensor:
    """y = A x; x: (..., nz, ny, nx) (2D: (..., ny, nx)); y: (..., nview, nv, nu)."""
    _check_tensor(x, "volume")
    lead = x.shape[:-len(geom.vol_shape)]
    y = torch.empty(tuple(lead) + geom.sino_shape, dtype=out_dtype or x.dtype, device=x.device)
    return forward_into(geom, x, y, projector, mode, stream)


def back(geom: Geometry, y: torch.Tensor, projector: str = "sf", mode: str = "proj",
         out_dtype: Optional[torch.dtype] = None, stream=None) -> torch.Tensor:
    """x = A^T y; y: (..., nview, nv, nu) (2D: (..., nview, nu)); x: (..., nz, ny, nx)."""
    _check_tensor(y, "sinogram")
    lead = y.shape[:-len(geom.sino_shape)]
    x = torch.empty(tuple(lead) + geom.vol_shape, dtype=out_dtype or y.dtype, device=y.device)
    return back_into(geom, y, x, projector, mode, stream)


def ramp_filter(geom: Geometry, y: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The pre-weighted discrete ramp filter of FBP (ct_ramp_filter), row by
    row; `out` may be `y` itself for an in-place filter."""
    _check_tensor(y, "sinogram")
    batch = _batch_of(y, geom.sino_shape, "sinogram")
    if out is None:
        out = torch.empty_like(y)
    _check_tensor(out, "output")
    if out.shape != y.shape:
        raise ValueError("output shape differs from the sinogram's")
    _check(load().ct_ramp_filter(geom.handle, DTYPES[y.dtype], y.data_ptr(), DTYPES[out.dtype], out.data_ptr(),
                                 batch, _stream_ptr(stream)))
    return out


def fbp(geom: Geometry, y: torch.Tensor, stream=None) -> torch.Tensor:
    """Filtered backprojection: the ramp filter, then the recon-mode
    (depth-weighted, voxel-driven) backprojection (Sec. 2.3)."""
    return back(geom, ramp_filter(geom, y, stream=stream), "voxel", mode="recon", stream=stream)


def back_dd_noalloc(geom: Geometry, y: torch.Tensor, out_dtype: Optional[torch.dtype] = None,
                    stream=None) -> torch.Tensor:
    """DD backprojection through ct_back_dd_noalloc: the library allocates
    nothing (its scratch is a fixed device array); the output tensor is
    allocated here by PyTorch."""
    _check_tensor(y, "sinogram")
    b = _batch_of(y, geom.sino_shape, "sinogram")
    lead = y.shape[:-len(geom.sino_shape)]
    x = torch.empty(tuple(lead) + geom.vol_shape, dtype=out_dtype or y.dtype, device=y.device)
    _check(load().ct_back_dd_noalloc(geom.handle, DTYPES[y.dtype], y.data_ptr(), DTYPES[x.dtype],
                                     x.data_ptr(), b, _stream_ptr(stream)))
    return x


def workspace_bytes(geom: Geometry, projector: str, direction: str, dtype: torch.dtype = torch.float32,
                    batch: int = 1, mode: str = "proj") -> int:
    """Pooled workspace (bytes) one forward ('fwd') or back ('back') call
    takes from the library on top of its input and output (ct_workspace_bytes)."""
    out = C.c_size_t(0)
    _check(load().ct_workspace_bytes(geom.handle, PROJECTORS[projector], MODES[mode],
                                     {"fwd": 0, "back": 1}[direction], DTYPES[dtype], int(batch), C.byref(out)))
    return int(out.value)


def workspace_limit(nbytes: int) -> None:
    """Cap what the current device's workspace pool keeps between calls
    (ct_workspace_limit)."""
    _check(load().ct_workspace_limit(int(nbytes)))


def workspace_usage(reset_high: bool = False):
    """(bytes the pool holds now, high-water mark of bytes in use since the
    last reset) for the current device (ct_workspace_usage)."""
    r, h = C.c_size_t(0), C.c_size_t(0)
    _check(load().ct_workspace_usage(C.byref(r), C.byref(h), 1 if reset_high else 0))
    return int(r.value), int(h.value)
