"""FP64 CPU oracle for CT forward projection and its adjoint (Sec. 2.3, Eq. 1-2).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
timed CPU-baseline leg may import this package.  The CUDA library never calls
it and shares no code with it; the two meet only in the seeded inputs of the
`workloads` module.

The arithmetic lives in `ct_oracle.c` (plain C, double precision, OpenMP over
independent outer loops), built on first use with the system C compiler.
Parity status per projector (what pins it in tests/test_oracle_*.py):
  ray-driven   brute-force all-pairs chord lengths, closed-form chords
  voxel-driven bilinear partition of unity, hand-derived single-voxel value
  DD           boundary partition, parallel-beam equality with exact row sums,
               3D partition with slab-method path lengths
  SF           trapezoid area identity, exact parallel-beam pixel projection,
               3D mass identity with the slab-method column chord
  SF-TT        trapezoid areas with the slab-method per-cell amplitude
hand-derived cone-beam weights off the mid-plane (SF, DD, SF-TT; flat and
curved), and for all the adjoint identity <Ax, y> = <x, A^T y>.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from workloads import GeometrySpec

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ct_oracle.c")
_LIB = os.path.join(_HERE, "libctoracle.so")
_lock = threading.Lock()
_lib = None

PROJECTORS = {"voxel": 0, "ray": 1, "dd": 2, "sf": 3, "sftt": 4}
KINDS = {"fan2d": 0, "circ3d": 1, "noncirc3d": 2}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("curved", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("nu", C.c_int), ("nv", C.c_int),
                ("du", C.c_double), ("dv", C.c_double),
                ("nview", C.c_int)] + [
        (n, C.POINTER(C.c_double)) for n in
        ("theta", "phi", "psi", "sad", "sdd", "x_src", "z_src",
         "x_ofst", "y_ofst", "z_ofst", "u_ofst", "v_ofst", "poses")]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            d = C.POINTER(C.c_double)
            lib.oracle_forward.argtypes = [P(_Desc), C.c_int, d, d, C.c_int]
            lib.oracle_back.argtypes = [P(_Desc), C.c_int, d, d, C.c_int]
            lib.oracle_back_voxels.argtypes = [P(_Desc), C.c_int, d, C.c_int, C.c_longlong,
                                               P(C.c_longlong), d]
            lib.oracle_footprint.argtypes = [P(_Desc), C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_int, P(C.c_int), P(C.c_int), d]
            lib.oracle_frame.argtypes = [P(_Desc), C.c_int, d]
            lib.oracle_project.argtypes = [P(_Desc), C.c_int, d, d]
            lib.oracle_cell_point.argtypes = [P(_Desc), C.c_int, C.c_int, C.c_int, d]
            lib.oracle_set_threads.argtypes = [C.c_int]
            lib.oracle_ramp_filter.argtypes = [P(_Desc), d, d, C.c_int]
            lib.oracle_back_recon.argtypes = [P(_Desc), d, d, C.c_int]
            lib.oracle_back_recon_proj.argtypes = [P(_Desc), C.c_int, d, d, C.c_int]
            lib.oracle_recon_dbeta.argtypes = [P(_Desc), C.c_int]
            lib.oracle_recon_dbeta.restype = C.c_double
            lib.oracle_max_threads.restype = C.c_int
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Geom:
    """Keeps the descriptor and the arrays it points to alive together."""

    def __init__(self, spec: GeometrySpec):
        self.spec = spec
        self.arrays = {}
        d = _Desc()
        d.kind = KINDS[spec.kind]
        d.curved = 1 if spec.det == "curved" else 0
        d.nx, d.ny, d.nz = spec.nx, spec.ny, spec.nz
        d.dx, d.dy, d.dz = spec.dx, spec.dy, spec.dz
        d.nu, d.nv = spec.nu, spec.nv
        d.du, d.dv = spec.du, spec.dv
        d.nview = spec.nview
        for n in ("theta", "phi", "psi", "sad", "sdd", "x_src", "z_src",
                  "x_ofst", "y_ofst", "z_ofst", "u_ofst", "v_ofst"):
            a = np.ascontiguousarray(spec.per_view(n), dtype=np.float64)
            self.arrays[n] = a
            setattr(d, n, _dptr(a))
        if spec.poses is not None:
            a = np.ascontiguousarray(np.asarray(spec.poses, dtype=np.float64).reshape(spec.nview, 12))
            self.arrays["poses"] = a
            d.poses = _dptr(a)
        else:
            d.poses = C.POINTER(C.c_double)()
        self.desc = d

    def ref(self):
        return C.byref(self.desc)


def _vol_shape(spec):
    return (1 if spec.kind == "fan2d" else spec.nz, spec.ny, spec.nx)


def _sino_shape(spec):
    return (spec.nview, 1 if spec.kind == "fan2d" else spec.nv, spec.nu)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def forward(spec: GeometrySpec, projector: str, vol: np.ndarray) -> np.ndarray:
    """y = A x in FP64.  vol: (nz, ny, nx) or (batch, nz, ny, nx)."""
    lib = _load()
    g = _Geom(spec)
    x = np.ascontiguousarray(vol, dtype=np.float64)
    squeeze = x.ndim == 3
    x = x.reshape((-1,) + _vol_shape(spec))
    y = np.zeros((x.shape[0],) + _sino_shape(spec))
    rc = lib.oracle_forward(g.ref(), PROJECTORS[projector], _dptr(x), _dptr(y), x.shape[0])
    if rc:
        raise RuntimeError("oracle footprint capacity exceeded")
    return y[0] if squeeze else y


def back(spec: GeometrySpec, projector: str, sino: np.ndarray) -> np.ndarray:
    """x = A^T y in FP64.  sino: (nview, nv, nu) or (batch, nview, nv, nu)."""
    lib = _load()
    g = _Geom(spec)
    y = np.ascontiguousarray(sino, dtype=np.float64)
    squeeze = y.ndim == 3
    y = y.reshape((-1,) + _sino_shape(spec))
    x = np.zeros((y.shape[0],) + _vol_shape(spec))
    rc = lib.oracle_back(g.ref(), PROJECTORS[projector], _dptr(y), _dptr(x), y.shape[0])
    if rc:
        raise RuntimeError("oracle footprint capacity exceeded")
    return x[0] if squeeze else x


def back_voxels(spec: GeometrySpec, projector: str, sino: np.ndarray,
                flat_index: np.ndarray) -> np.ndarray:
    """(A^T y) at the listed flat voxel indices (k*ny + j)*nx + i."""
    lib = _load()
    g = _Geom(spec)
    y = np.ascontiguousarray(sino, dtype=np.float64)
    squeeze = y.ndim == 3
    y = y.reshape((-1,) + _sino_shape(spec))
    sel = np.ascontiguousarray(flat_index, dtype=np.int64)
    out = np.zeros((y.shape[0], sel.size))
    rc = lib.oracle_back_voxels(g.ref(), PROJECTORS[projector], _dptr(y), y.shape[0],
                                sel.size, sel.ctypes.data_as(C.POINTER(C.c_longlong)), _dptr(out))
    if rc:
        raise RuntimeError("oracle footprint capacity exceeded")
    return out[0] if squeeze else out


def footprint(spec: GeometrySpec, projector: str, view: int, i: int, j: int, k: int):
    """Cells (a, b) and weights of voxel (i, j, k) in one view."""
    lib = _load()
    g = _Geom(spec)
    cap = 8192
    a = np.zeros(cap, dtype=np.int32)
    b = np.zeros(cap, dtype=np.int32)
    w = np.zeros(cap)
    n = lib.oracle_footprint(g.ref(), PROJECTORS[projector], view, i, j, k, cap,
                             a.ctypes.data_as(C.POINTER(C.c_int)),
                             b.ctypes.data_as(C.POINTER(C.c_int)), _dptr(w))
    if n < 0:
        raise RuntimeError("footprint too large")
    return a[:n].copy(), b[:n].copy(), w[:n].copy()


def frame(spec: GeometrySpec, view: int) -> dict:
    """The view's source, detector centre, axes and derived distances."""
    g = _Geom(spec)
    out = np.zeros(18)
    _load().oracle_frame(g.ref(), view, _dptr(out))
    return {"s": out[0:3], "c": out[3:6], "eu": out[6:9], "ev": out[9:12],
            "n": out[12:15], "D": out[15], "u0": out[16], "h0": out[17]}


def project(spec: GeometrySpec, view: int, X) -> np.ndarray:
    """Detector (u, v) in mm of world point X."""
    g = _Geom(spec)
    x = np.ascontiguousarray(X, dtype=np.float64)
    uv = np.zeros(2)
    _load().oracle_project(g.ref(), view, _dptr(x), _dptr(uv))
    return uv


def cell_point(spec: GeometrySpec, view: int, a: int, b: int) -> np.ndarray:
    """World position of the centre of detector cell (a, b)."""
    g = _Geom(spec)
    P = np.zeros(3)
    _load().oracle_cell_point(g.ref(), view, a, b, _dptr(P))
    return P


def ramp_filter(spec: GeometrySpec, sino: np.ndarray) -> np.ndarray:
    """Pre-weighted, ramp-filtered projections of the "recon" mode (FBP,
    Sec. 2.3).  sino: (nview, nv, nu) or (batch, nview, nv, nu)."""
    lib = _load()
    g = _Geom(spec)
    y = np.ascontiguousarray(sino, dtype=np.float64)
    squeeze = y.ndim == 3
    y = y.reshape((-1,) + _sino_shape(spec))
    q = np.zeros_like(y)
    lib.oracle_ramp_filter(g.ref(), _dptr(y), _dptr(q), y.shape[0])
    return q[0] if squeeze else q


def back_recon(spec: GeometrySpec, q: np.ndarray, projector: str = "voxel") -> np.ndarray:
    """Recon-mode (depth-weighted) backprojection of filtered projections q:
    the second half of FBP, with the voxel-driven bilinear interpolation or
    the normalised DD / SF footprints."""
    lib = _load()
    g = _Geom(spec)
    y = np.ascontiguousarray(q, dtype=np.float64)
    squeeze = y.ndim == 3
    y = y.reshape((-1,) + _sino_shape(spec))
    x = np.zeros((y.shape[0],) + _vol_shape(spec))
    lib.oracle_back_recon_proj(g.ref(), PROJECTORS[projector], _dptr(y), _dptr(x), y.shape[0])
    return x[0] if squeeze else x


def fbp(spec: GeometrySpec, sino: np.ndarray, projector: str = "voxel") -> np.ndarray:
    """Filtered backprojection: back_recon(ramp_filter(sino))."""
    return back_recon(spec, ramp_filter(spec, sino), projector)


def recon_dbeta(spec: GeometrySpec, view: int) -> float:
    """The view's share of the gantry angle used by the recon mode."""
    return float(_load().oracle_recon_dbeta(_Geom(spec).ref(), view))
