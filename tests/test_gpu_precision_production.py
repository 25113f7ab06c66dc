"""Half storage on the code paths the benchmark workloads take.

The ragged geometries of test_gpu_precision.py (nz = 21, axial footprints of
about 0.6 rows) never reach two branches that every circular benchmark size
takes: the forward's z-major vector loads (four voxels per load, nz a
multiple of 4) and the axial footprint shorter than half a row.  These cases
use scaled copies of the 256^3 / 360-view flat workload and of the curved
984-view workload, which keep the full sizes' footprints in cells and have nz
a multiple of 4, plus a sampled check of the 256^3 workload at full size.

Bounds: see test_gpu_precision.py.  A storage rounding with unit roundoff u
costs at most u relative error (A and the data are non-negative); FP32
arithmetic adds ~1e-5.  Measured errors are printed per case."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import TOL_F16, rel_l2

pytestmark = pytest.mark.gpu
T = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
ARITH = 2e-5
CASES = [("f16", "f16", 2.0 ** -10 + ARITH), ("f16", "f32", 2.0 ** -11 + ARITH),
         ("f32", "f16", 2.0 ** -11 + ARITH), ("bf16", "f32", 2.0 ** -8 + ARITH),
         ("f32", "bf16", 2.0 ** -8 + ARITH), ("bf16", "bf16", 2.0 ** -7 + ARITH)]

GEOMS = {
    # 64^3 of 2 mm, 90 views, 128 x 96 cells of 3.2 mm: axial footprint 0.86 rows
    "circ-flat-64": lambda: W.scaled(W.circ3d_256(), 64, 90),
    # 128^2 x 32, 123 views, curved 222 x 16: axial footprint 0.46 rows
    "circ-curved-128": lambda: W.scaled(W.circ3d_curved(), 128, 123),
}


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


@functools.lru_cache(maxsize=None)
def _spec(name):
    spec = GEOMS[name]()
    assert spec.nz % 4 == 0
    return spec


@functools.lru_cache(maxsize=None)
def _inputs(name):
    spec = _spec(name)
    return W.phantom(spec, seed=11), W.random_sino(spec, seed=11)[0]


@functools.lru_cache(maxsize=None)
def _reference(name, proj):
    spec = _spec(name)
    x, s = _inputs(name)
    return oracle.forward(spec, proj, x), oracle.back(spec, proj, s)


def _projectors(name):
    spec = _spec(name)
    return ["voxel", "ray", "dd", "sf"] + (["sftt"] if spec.det == "flat" else [])


PARAMS = [(n, p, tin, tout, b) for n in GEOMS for p in _projectors(n) for (tin, tout, b) in CASES]


@pytest.mark.parametrize("name,proj,tin,tout,bound", PARAMS,
                         ids=[f"{n}-{p}-{i}-{o}" for n, p, i, o, _ in PARAMS])
def test_half_storage_on_production_paths(ct, report, name, proj, tin, tout, bound):
    assert bound <= TOL_F16 or "bf16" in (tin, tout)
    spec = _spec(name)
    x, s = _inputs(name)
    y_ref, x_ref = _reference(name, proj)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).to(T[tin]).cuda(), proj, out_dtype=T[tout])
    xb = ct.back(g, torch.as_tensor(s, dtype=torch.float32).to(T[tin]).cuda(), proj, out_dtype=T[tout])
    torch.cuda.synchronize()
    e_fwd = rel_l2(y.float().cpu().numpy(), y_ref)
    e_back = rel_l2(xb.float().cpu().numpy(), x_ref)
    report(f"{name} {proj} {tin}->{tout}: forward {e_fwd:.2e}, back {e_back:.2e} (bound {bound:.2e})")
    assert e_fwd <= bound and e_back <= bound, (e_fwd, e_back)


def _sample_voxels(spec, n, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(spec.n_vox, size=n, replace=False)


@pytest.mark.parametrize("proj", ["sf", "dd"])
@pytest.mark.parametrize("tin,tout,bound", [("f16", "f16", 2.0 ** -10 + ARITH),
                                            ("bf16", "bf16", 2.0 ** -7 + ARITH)])
def test_circ3d_256_full_size_half_storage(ct, report, proj, tin, tout, bound):
    """The 256^3 / 360-view workload at full size in half storage: the
    forward on four views and the back at 300 sampled voxels, both against
    the FP64 oracle on the unrounded inputs."""
    spec = W.circ3d_256()
    x = W.phantom(spec, seed=0)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).to(T[tin]).cuda(), proj, out_dtype=T[tout])
    torch.cuda.synchronize()
    views = [0, 47, 133, 271]
    e_fwd = rel_l2(y[views].float().cpu().numpy(), oracle.forward(spec.subset(views), proj, x))
    s = W.random_sino(spec, seed=5)[0]
    xb = ct.back(g, torch.as_tensor(s, dtype=torch.float32).to(T[tin]).cuda(), proj, out_dtype=T[tout])
    torch.cuda.synchronize()
    sel = _sample_voxels(spec, 300, 6)
    e_back = rel_l2(xb.float().cpu().numpy().ravel()[sel], oracle.back_voxels(spec, proj, s, sel))
    report(f"circ3d_256 full size {proj} {tin}->{tout}: forward {e_fwd:.2e}, back {e_back:.2e}")
    assert e_fwd <= bound and e_back <= bound, (e_fwd, e_back)
