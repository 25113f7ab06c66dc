"""ct_back_dd_noalloc: the DD backprojection for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).
Such callers include a service whose device memory belongs to another
allocator, a plug-in inside a host application that forbids allocation after
start-up, and a latency-critical path that must not risk an allocation.

It must give what ct_back(CT_DD) gives, bit for bit, on consecutive calls
that reuse the same scratch array: the two run the same kernels on the same
inputs.  Collected last so that a failure here comes after every other test
has run."""
import ctypes as C
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from gpu_util import ragged

pytestmark = pytest.mark.gpu
T = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _sino(spec, seed, batch, dtype):
    shape = (spec.nview, spec.nu) if spec.kind == "fan2d" else spec.sino_shape
    ys = [W.random_sino(spec, seed=seed + b)[0].reshape(shape) for b in range(batch)]
    y = np.stack(ys) if batch > 1 else ys[0]
    return torch.as_tensor(y, dtype=torch.float32).to(dtype).cuda()


@pytest.mark.parametrize("kind,det", [("circ3d", "flat"), ("circ3d", "curved"), ("fan2d", "flat"),
                                      ("noncirc3d", "flat")])
@pytest.mark.parametrize("tin,tout", [("f32", "f32"), ("f16", "f32"), ("bf16", "bf16"), ("f16", "f16")])
@pytest.mark.parametrize("batch", [1, 2])
def test_noalloc_equals_ct_back_on_two_calls(ct, kind, det, tin, tout, batch):
    spec = ragged(kind, det, seed=21)
    g = ct.Geometry.from_spec(spec)
    for seed in (1, 5):  # the second call finds the first call's scratch contents
        y = _sino(spec, seed, batch, T[tin])
        ref = ct.back(g, y, "dd", out_dtype=T[tout])
        got = ct.back_dd_noalloc(g, y, out_dtype=T[tout])
        torch.cuda.synchronize()
        assert got.dtype == ref.dtype and got.shape == ref.shape
        assert torch.equal(got, ref)


def test_noalloc_wide_noncircular_footprints(ct):
    """Footprints wider than the footprint kernels' 8 cells take the general
    gather (no scratch) in both entry points."""
    spec = W.scaled(W.noncirc3d_saddle(), 24, 7)
    spec = dataclasses.replace(spec, du=spec.du / 4, nu=spec.nu * 4)
    g = ct.Geometry.from_spec(spec)
    for seed in (2, 3):
        y = _sino(spec, seed, 1, torch.float32)
        assert torch.equal(ct.back_dd_noalloc(g, y), ct.back(g, y, "dd"))


def test_noalloc_rejects_host_pointers(ct):
    """A host buffer is an argument error reported before any launch."""
    spec = ragged("circ3d", "flat", seed=21)
    g = ct.Geometry.from_spec(spec)
    lib = ct.load()
    y_host = torch.zeros(spec.sino_shape)
    x_dev = torch.empty(spec.vol_shape, device="cuda")
    rc = lib.ct_back_dd_noalloc(g.handle, 0, C.c_void_p(y_host.data_ptr()), 0, C.c_void_p(x_dev.data_ptr()),
                                1, None)
    assert rc == 1 and lib.ct_last_error().decode().startswith("input: not")
    y_dev = torch.zeros(spec.sino_shape, device="cuda")
    x_host = torch.empty(spec.vol_shape)
    rc = lib.ct_back_dd_noalloc(g.handle, 0, C.c_void_p(y_dev.data_ptr()), 0, C.c_void_p(x_host.data_ptr()),
                                1, None)
    assert rc == 1 and lib.ct_last_error().decode().startswith("output: not")
    torch.cuda.synchronize()


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
