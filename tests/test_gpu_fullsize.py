"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark times, on outputs the oracle can afford: the
forward projection of a few views (a view subset is a geometry of its own)
and the backprojection at sampled voxels (all views)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import TOL_F16, TOL_F32, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _sample_voxels(spec, n, seed):
    rng = np.random.default_rng(seed)
    return rng.choice(spec.n_vox, size=n, replace=False)


@pytest.mark.parametrize("proj", ["sf", "dd", "ray", "voxel"])
def test_circ3d_256_full_size(ct, proj):
    spec = W.circ3d_256()
    x = W.phantom(spec, seed=0)
    g = ct.Geometry.from_spec(spec)
    xd = torch.as_tensor(x, dtype=torch.float32).cuda()
    y = ct.forward(g, xd, proj)
    xb = ct.back(g, y, proj)
    torch.cuda.synchronize()
    views = [0, 47, 133, 271]
    y_ref = oracle.forward(spec.subset(views), proj, x)
    assert rel_l2(y[views].cpu().numpy(), y_ref) <= TOL_F32
    sel = _sample_voxels(spec, 300, 1)
    xb_ref = oracle.back_voxels(spec, proj, y.double().cpu().numpy(), sel)
    assert rel_l2(xb.cpu().numpy().ravel()[sel], xb_ref) <= TOL_F32


def test_circ3d_curved_full_size_dd(ct):
    spec = W.circ3d_curved()
    x = W.phantom(spec, seed=2)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).cuda(), "dd")
    torch.cuda.synchronize()
    views = [5, 500]
    assert rel_l2(y[views].cpu().numpy(), oracle.forward(spec.subset(views), "dd", x)) <= TOL_F32
    s = W.random_sino(spec, seed=2)[0].astype(np.float32)
    xb = ct.back(g, torch.as_tensor(s).cuda(), "dd")
    sel = _sample_voxels(spec, 200, 2)
    ref = oracle.back_voxels(spec, "dd", s.astype(np.float64), sel)
    assert rel_l2(xb.cpu().numpy().ravel()[sel], ref) <= TOL_F32


@pytest.mark.parametrize("dtype,bound", [(torch.float32, TOL_F32), (torch.float16, TOL_F16)])
def test_noncirc_512_full_size_sf(ct, dtype, bound):
    spec = W.noncirc3d_saddle()
    x = W.phantom(spec, seed=0)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x, dtype=dtype).cuda(), "sf")
    torch.cuda.synchronize()
    views = [123]
    assert rel_l2(y[views].float().cpu().numpy(), oracle.forward(spec.subset(views), "sf", x)) <= bound
    sel = _sample_voxels(spec, 100, 3)
    yy = y.float()
    xb = ct.back(g, y, "sf")
    ref = oracle.back_voxels(spec, "sf", yy.double().cpu().numpy(), sel)
    assert rel_l2(xb.float().cpu().numpy().ravel()[sel], ref) <= bound


def test_fan2d_small_full_size_ray_forward_voxel_back(ct):
    """The fan-beam workload in full: ray-driven forward of the phantom and
    voxel-driven backprojection of its sinogram, every output element."""
    spec = W.fan2d_small()
    x = W.phantom(spec, seed=0)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x.reshape(spec.ny, spec.nx), dtype=torch.float32).cuda(), "ray")
    torch.cuda.synchronize()
    y_ref = oracle.forward(spec, "ray", x)
    assert rel_l2(y.cpu().numpy().reshape(y_ref.shape), y_ref) <= TOL_F32
    xb = ct.back(g, y, "voxel")
    xb_ref = oracle.back(spec, "voxel", y.double().cpu().numpy().reshape(y_ref.shape))
    assert rel_l2(xb.cpu().numpy().reshape(xb_ref.shape), xb_ref) <= TOL_F32


def test_noncirc_512_full_size_dd(ct):
    spec = W.noncirc3d_saddle()
    x = W.phantom(spec, seed=4)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).cuda(), "dd")
    torch.cuda.synchronize()
    views = [3, 250]
    assert rel_l2(y[views].cpu().numpy(), oracle.forward(spec.subset(views), "dd", x)) <= TOL_F32
    sel = _sample_voxels(spec, 100, 4)
    xb = ct.back(g, y, "dd")
    ref = oracle.back_voxels(spec, "dd", y.double().cpu().numpy(), sel)
    assert rel_l2(xb.cpu().numpy().ravel()[sel], ref) <= TOL_F32


@pytest.mark.parametrize("workload,proj", [("circ3d_256", "sf"), ("circ3d_256", "dd"), ("noncirc3d_saddle", "sf")])
def test_full_size_adjoint_identity(ct, workload, proj):
    """<A x, y> = <x, A^T y> at the benchmark sizes, on the code paths the
    benchmark times (the forward's axial sweep with vector column loads, the
    back's packed row filter; the footprint kernels in non-circular
    geometry), with the dot products taken in FP64."""
    spec = getattr(W, workload)()
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(7)
    x = torch.rand(g.vol_shape, generator=gen, device="cuda")
    y = torch.rand(g.sino_shape, generator=gen, device="cuda")
    ax = ct.forward(g, x, proj)
    aty = ct.back(g, y, proj)
    lhs = float((ax.double() * y.double()).sum())
    rhs = float((x.double() * aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
