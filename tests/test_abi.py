"""The C ABI without a GPU: the library loads, exports every function that
include/ctproj.h declares, and rejects malformed requests on the host before
touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for h in sorted(os.listdir(HEADER_DIR)):
        if h.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ct_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2503_16741_gb300 import build
    return C.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ct_geometry_create", "ct_geometry_destroy", "ct_forward", "ct_back", "ct_last_error"):
        assert f in names


def test_every_declared_function_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def _desc(**over):
    from paper_2503_16741_gb300.binding import _Desc
    d = _Desc()
    d.kind, d.det = 1, 0
    d.nx = d.ny = d.nz = 8
    d.dx = d.dy = d.dz = 1.0
    d.nu, d.nv, d.du, d.dv, d.nview = 16, 8, 1.0, 1.0, 4
    keep = []
    for k, v in over.items():
        if isinstance(v, (list, tuple, np.ndarray)):
            a = np.ascontiguousarray(v, dtype=np.float64)
            keep.append(a)
            setattr(d, k, a.ctypes.data_as(C.POINTER(C.c_double)))
            setattr(d, "n_" + k, a.size)
        else:
            setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("over,status", [
    (dict(nx=0), 1),                                   # empty volume
    (dict(kind=7), 1),                                 # unknown geometry kind
    (dict(kind=2, det=1), 2),                          # curved non-circular: unsupported
    (dict(kind=0, nz=4), 1),                           # fan beam with several slices
    (dict(du=-1.0), 1),                                # negative cell size
    (dict(theta=[0.0, 1.0, 2.0]), 1),                  # per-view vector of wrong length
])
def test_create_rejects_bad_descriptions(lib, over, status):
    base = dict(sad=[500.0], sdd=[1000.0], theta=[0.0, 1.0, 2.0, 3.0])
    base.update(over)
    d, keep = _desc(**base)
    h = C.c_void_p()
    lib.ct_geometry_create.argtypes = [C.c_void_p, C.c_void_p]
    lib.ct_last_error.restype = C.c_char_p
    rc = lib.ct_geometry_create(C.byref(d), C.byref(h))
    assert rc == status
    assert h.value is None
    assert lib.ct_last_error().decode() != ""


def test_calls_on_a_null_geometry_are_rejected(lib):
    lib.ct_forward.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                               C.c_void_p, C.c_int, C.c_void_p]
    lib.ct_back.argtypes = lib.ct_forward.argtypes
    assert lib.ct_forward(None, 3, 0, 0, None, 0, None, 1, None) == 1
    assert lib.ct_back(None, 3, 0, 0, None, 0, None, 1, None) == 1
    lib.ct_geometry_destroy.argtypes = [C.c_void_p]
    assert lib.ct_geometry_destroy(None) == 0


def test_geometry_requires_sad_and_sdd(lib):
    """The header's rule (sad and sdd must be given) holds in the binding too:
    no silent default distances."""
    from paper_2503_16741_gb300.binding import Geometry
    with pytest.raises(TypeError, match="sad and sdd"):
        Geometry("circ3d", "flat", 8, 8, 8, 1.0, 1.0, 1.0, 16, 8, 1.0, 1.0, 4, theta=0.0)
    with pytest.raises(TypeError, match="sad and sdd"):
        Geometry("circ3d", "flat", 8, 8, 8, 1.0, 1.0, 1.0, 16, 8, 1.0, 1.0, 4, sad=500.0)
