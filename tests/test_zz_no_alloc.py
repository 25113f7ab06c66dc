"""ct_back_dd_noalloc: the DD backprojection for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
It must give what ct_back(CT_DD) gives, on consecutive calls that reuse the
same scratch array.  Collected last so that a failure here comes after every
other test has run."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from gpu_util import TOL_F32, ragged, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _noalloc(ct, g, y):
    lib = ct.load()
    x = torch.empty((g.nz, g.ny, g.nx) if not g.is2d else (g.ny, g.nx), device="cuda")
    rc = lib.ct_back_dd_noalloc(g.handle, 0, C.c_void_p(y.data_ptr()), 0, C.c_void_p(x.data_ptr()), 1,
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.ct_last_error().decode()
    return x


@pytest.mark.parametrize("kind,det", [("circ3d", "flat"), ("circ3d", "curved"), ("fan2d", "flat")])
def test_noalloc_matches_ct_back_on_two_calls(ct, kind, det):
    spec = ragged(kind, det, seed=21)
    g = ct.Geometry.from_spec(spec)
    shape = (spec.nview, spec.nu) if kind == "fan2d" else spec.sino_shape
    for seed in (1, 2):  # the second call finds the first call's scratch contents
        y = torch.as_tensor(W.random_sino(spec, seed=seed)[0].reshape(shape), dtype=torch.float32).cuda()
        ref = ct.back(g, y, "dd")
        got = _noalloc(ct, g, y)
        torch.cuda.synchronize()
        assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) <= TOL_F32


def test_noalloc_rejects_sizes_beyond_its_scratch(ct):
    spec = W.GeometrySpec("circ3d", "flat", 8, 8, 8, 1.0, 1.0, 1.0, 1024, 1024, 0.3, 0.3, 17,
                          theta=np.linspace(0, 6, 17), sad=300.0, sdd=600.0)
    g = ct.Geometry.from_spec(spec)
    lib = ct.load()
    y = torch.zeros((17, 1024, 1024), device="cuda")
    x = torch.empty((8, 8, 8), device="cuda")
    rc = lib.ct_back_dd_noalloc(g.handle, 0, C.c_void_p(y.data_ptr()), 0, C.c_void_p(x.data_ptr()), 1, None)
    assert rc == 1
    assert "exceeds the static scratch" in lib.ct_last_error().decode()
