"""Recon mode (filtered backprojection, Sec. 2.3) on the GPU against the
FP64 oracle: the pre-weighted ramp filter row by row, the depth-weighted
voxel-driven backprojection, and FBP end to end, on the ragged geometries
(uneven view angles, every offset set) of all kinds and detectors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import GEOMS, TOL_F32, ragged, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _sino_shape(spec):
    return (spec.nview, spec.nu) if spec.kind == "fan2d" else (spec.nview, spec.nv, spec.nu)


@pytest.mark.parametrize("kind,det", GEOMS)
@pytest.mark.parametrize("data", ["projection", "random"])
def test_ramp_filter_matches_oracle(ct, kind, det, data):
    spec = ragged(kind, det, seed=50)
    if data == "projection":
        y = oracle.forward(spec, "sf", W.phantom(spec, seed=1))
    else:
        y = W.random_sino(spec, seed=2)[0]
    ref = oracle.ramp_filter(spec, y)
    g = ct.Geometry.from_spec(spec)
    q = ct.ramp_filter(g, torch.as_tensor(y.reshape(_sino_shape(spec)), dtype=torch.float32).cuda())
    assert rel_l2(q.cpu().numpy().reshape(ref.shape), ref) <= TOL_F32


@pytest.mark.parametrize("proj", ["voxel", "dd", "sf"])
@pytest.mark.parametrize("kind,det", GEOMS)
def test_recon_backprojection_matches_oracle(ct, kind, det, proj):
    spec = ragged(kind, det, seed=51)
    q = oracle.ramp_filter(spec, oracle.forward(spec, "dd", W.phantom(spec, seed=3)))
    ref = oracle.back_recon(spec, q, proj)
    g = ct.Geometry.from_spec(spec)
    x = ct.back(g, torch.as_tensor(q.reshape(_sino_shape(spec)), dtype=torch.float32).cuda(), proj,
                mode="recon")
    assert rel_l2(x.cpu().numpy().reshape(ref.shape), ref) <= TOL_F32


@pytest.mark.parametrize("kind,det", GEOMS)
def test_fbp_matches_oracle_and_filters_in_place(ct, kind, det):
    spec = ragged(kind, det, seed=52)
    y = oracle.forward(spec, "sf", W.phantom(spec, seed=4))
    ref = oracle.fbp(spec, y)
    g = ct.Geometry.from_spec(spec)
    yd = torch.as_tensor(y.reshape(_sino_shape(spec)), dtype=torch.float32).cuda()
    x = ct.fbp(g, yd)
    assert rel_l2(x.cpu().numpy().reshape(ref.shape), ref) <= TOL_F32
    q = ct.ramp_filter(g, yd)
    yd2 = yd.clone()
    assert torch.equal(ct.ramp_filter(g, yd2, out=yd2), q)


def test_fbp_reconstructs_a_z_invariant_gaussian(ct):
    """The library's FDK on the oracle pin's object: a Gaussian cylinder from
    closed-form projections, reconstructed at every slice to 0.5 % of its peak."""
    from test_oracle_fbp import _gauss_cyl_sino, _uneven_angles
    nx, nz, nview, mu, sigma, c = 48, 48, 180, 0.02, 5.0, (8.0, -5.0)
    for det in ("flat", "curved"):
        spec = W.GeometrySpec("circ3d", det, nx, nx, nz, 1.0, 1.0, 1.0, 160, 176, 0.8, 1.0, nview,
                              theta=_uneven_angles(nview), sad=200.0, sdd=400.0, u_ofst=8.0, v_ofst=15.0)
        y = _gauss_cyl_sino(spec, (c[0], c[1], 0.0), sigma, mu)
        x = ct.fbp(ct.Geometry.from_spec(spec), torch.as_tensor(y, dtype=torch.float32).cuda()).cpu().numpy()
        g_ = np.arange(nx) - 0.5 * (nx - 1)
        yy, xx = np.meshgrid(g_, g_, indexing="ij")
        ref = mu * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / (2 * sigma ** 2))
        roi = np.hypot(xx, yy) < 20
        assert max(np.abs(x[k] - ref)[roi].max() for k in range(nz)) < 0.005 * mu


def test_half_storage_fbp(ct):
    """FP16 projections: the GPU's FBP of the stored values matches the FP64
    FBP of the same rounded values to the FP32 bound; the storage rounding
    itself costs more than for the projector pair, because the ramp filter
    amplifies the rounding noise (here about 2.5x the FP16 unit roundoff
    2^-11; the bound below is 5x it)."""
    spec = ragged("circ3d", "flat", seed=53)
    y = oracle.forward(spec, "sf", W.phantom(spec, seed=5))
    yh = torch.as_tensor(y, dtype=torch.float32).cuda().half()
    y_rounded = yh.double().cpu().numpy()
    g = ct.Geometry.from_spec(spec)
    q = ct.ramp_filter(g, yh, out=torch.empty(yh.shape, dtype=torch.float32, device="cuda"))
    x = ct.back(g, q, "voxel", mode="recon")
    assert rel_l2(x.cpu().numpy(), oracle.fbp(spec, y_rounded)) <= TOL_F32
    storage = rel_l2(oracle.fbp(spec, y_rounded), oracle.fbp(spec, y))
    assert storage <= 5 * 2.0 ** -11, storage


def test_recon_mode_is_a_backprojection_of_voxel_dd_or_sf(ct):
    spec = ragged("circ3d", "flat", seed=54)
    g = ct.Geometry.from_spec(spec)
    x = torch.rand(spec.vol_shape, device="cuda")
    y = torch.rand(spec.sino_shape, device="cuda")
    for proj in ("voxel", "sf"):
        with pytest.raises(ct.CTError):
            ct.forward(g, x, proj, mode="recon")
    for proj in ("ray", "sftt"):
        with pytest.raises(ct.CTError):
            ct.back(g, y, proj, mode="recon")


@pytest.mark.parametrize("proj", ["dd", "sf"])
def test_footprint_fbp_reconstructs_the_gaussian_cylinder(ct, proj):
    from test_oracle_fbp import _gauss_cyl_sino, _uneven_angles
    nx, nz, nview, mu, sigma, c = 48, 24, 180, 0.02, 5.0, (8.0, -5.0)
    spec = W.GeometrySpec("circ3d", "flat", nx, nx, nz, 1.0, 1.0, 1.0, 160, 96, 0.8, 1.0, nview,
                          theta=_uneven_angles(nview), sad=200.0, sdd=400.0, u_ofst=8.0, v_ofst=15.0)
    y = _gauss_cyl_sino(spec, (c[0], c[1], 0.0), sigma, mu)
    g = ct.Geometry.from_spec(spec)
    q = ct.ramp_filter(g, torch.as_tensor(y, dtype=torch.float32).cuda())
    x = ct.back(g, q, proj, mode="recon").cpu().numpy()
    ref_o = oracle.fbp(spec, y, proj)
    assert rel_l2(x, ref_o) <= TOL_F32
    g_ = np.arange(nx) - 0.5 * (nx - 1)
    yy, xx = np.meshgrid(g_, g_, indexing="ij")
    ref = mu * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / (2 * sigma ** 2))
    roi = np.hypot(xx, yy) < 20
    assert max(np.abs(x[k] - ref)[roi].max() for k in range(nz)) < 0.01 * mu


def test_fbp_batches_are_independent(ct):
    spec = ragged("circ3d", "curved", seed=55)
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(11)
    y = torch.rand((2, 3) + spec.sino_shape, generator=gen, device="cuda")
    x = ct.fbp(g, y)
    for b in range(2):
        for c in range(3):
            assert torch.equal(x[b, c], ct.fbp(g, y[b, c].contiguous()))
    q = ct.ramp_filter(g, y)
    for proj in ("dd", "sf"):
        xb = ct.back(g, q, proj, mode="recon")
        assert torch.equal(xb[1, 2], ct.back(g, q[1, 2].contiguous(), proj, mode="recon"))


@pytest.mark.parametrize("det", ["flat", "curved"])
@pytest.mark.parametrize("nu", [1000, 4097, 16384])
def test_ramp_filter_wide_rows(ct, det, nu):
    """Rows far wider than one thread block's outputs, up to the widest row the
    filter takes (16384 cells: its shared-memory row and taps nearly fill a
    block's 227 KB), even and odd widths."""
    spec = W.GeometrySpec("circ3d", det, 16, 16, 4, 1.0, 1.0, 1.0, nu, 3, 16.0 * 40 / nu, 1.0, 3,
                          theta=np.array([0.0, 2.0, 4.0]), sad=300.0, sdd=600.0, u_ofst=1.3, v_ofst=0.4)
    y = W.random_sino(spec, seed=9)[0]
    ref = oracle.ramp_filter(spec, y)
    g = ct.Geometry.from_spec(spec)
    q = ct.ramp_filter(g, torch.as_tensor(y, dtype=torch.float32).cuda())
    assert rel_l2(q.cpu().numpy(), ref) <= TOL_F32
