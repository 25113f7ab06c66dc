"""GPU (CUDA, through the C ABI) versus the FP64 oracle on seeded inputs.

FP32 storage must match within relative L2 1e-5 (the bound the FP32 path is
held to); the pair must satisfy the adjoint identity in FP32 to 1e-5."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import GEOMS, PROJECTORS, TOL_F32, ragged, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _gpu(ct, spec):
    return ct.Geometry.from_spec(spec)


def ct_vol_shape(spec):
    return (spec.ny, spec.nx) if spec.kind == "fan2d" else (spec.nz, spec.ny, spec.nx)


def ct_sino_shape(spec):
    return (spec.nview, spec.nu) if spec.kind == "fan2d" else (spec.nview, spec.nv, spec.nu)


@pytest.mark.parametrize("proj", PROJECTORS)
@pytest.mark.parametrize("kind,det", GEOMS)
def test_forward_matches_oracle(ct, kind, det, proj):
    spec = ragged(kind, det)
    x = W.phantom(spec, seed=1)
    ref = oracle.forward(spec, proj, x)
    g = _gpu(ct, spec)
    y = ct.forward(g, torch.as_tensor(x.reshape(ct_vol_shape(spec)), dtype=torch.float32).cuda(), proj)
    torch.cuda.synchronize()
    err = rel_l2(y.cpu().numpy().reshape(ref.shape), ref)
    assert np.linalg.norm(ref) > 0
    assert err <= TOL_F32, f"{kind}/{det}/{proj}: rel L2 {err:.3e}"


@pytest.mark.parametrize("proj", PROJECTORS)
@pytest.mark.parametrize("kind,det", GEOMS)
def test_back_matches_oracle(ct, kind, det, proj):
    spec = ragged(kind, det)
    y = W.random_sino(spec, seed=2)[0]
    ref = oracle.back(spec, proj, y)
    g = _gpu(ct, spec)
    x = ct.back(g, torch.as_tensor(y.reshape(ct_sino_shape(spec)), dtype=torch.float32).cuda(), proj)
    torch.cuda.synchronize()
    err = rel_l2(x.cpu().numpy().reshape(ref.shape), ref)
    assert err <= TOL_F32, f"{kind}/{det}/{proj}: rel L2 {err:.3e}"


@pytest.mark.parametrize("proj", PROJECTORS)
@pytest.mark.parametrize("kind,det", GEOMS)
def test_adjoint_identity_fp32(ct, kind, det, proj):
    spec = ragged(kind, det, seed=3)
    g = _gpu(ct, spec)
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand(ct_vol_shape(spec), generator=gen, device="cuda")
    y = torch.rand(ct_sino_shape(spec), generator=gen, device="cuda")
    Ax = ct.forward(g, x, proj)
    Aty = ct.back(g, y, proj)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    assert abs(lhs - rhs) <= TOL_F32 * abs(lhs), f"{lhs} vs {rhs}"


@pytest.mark.parametrize("kind", ["circ3d", "noncirc3d"])
@pytest.mark.parametrize("proj", PROJECTORS)
def test_batch_items_independent_and_deterministic(ct, proj, kind):
    spec = ragged(kind, "flat", seed=4)
    g = _gpu(ct, spec)
    gen = torch.Generator(device="cuda").manual_seed(9)
    x = torch.rand((2, 3) + ct_vol_shape(spec), generator=gen, device="cuda")
    y = ct.forward(g, x, proj)
    for b in range(2):
        for c in range(3):
            assert torch.equal(y[b, c], ct.forward(g, x[b, c].contiguous(), proj))
    assert torch.equal(y, ct.forward(g, x, proj))
    s = torch.rand((2,) + ct_sino_shape(spec), generator=gen, device="cuda")
    xb = ct.back(g, s, proj)
    assert torch.equal(xb[1], ct.back(g, s[1].contiguous(), proj))


@pytest.mark.parametrize("proj", PROJECTORS)
def test_view_subset_equals_slice(ct, proj):
    """Ordered subsets: a geometry of selected views gives those views."""
    spec = ragged("noncirc3d", "flat", seed=6)
    x = torch.as_tensor(W.phantom(spec, seed=2), dtype=torch.float32).cuda()
    full = ct.forward(_gpu(ct, spec), x, proj)
    views = [0, 5, 17, 22]
    sub = ct.forward(_gpu(ct, spec.subset(views)), x, proj)
    assert torch.equal(sub, full[views])


@pytest.mark.parametrize("kind", ["circ3d", "noncirc3d"])
def test_degenerate_sizes(ct, kind):
    """Single voxel, single cell, single view (tilted in the non-circular case)."""
    kw = dict(phi=0.08, psi=-0.03) if kind == "noncirc3d" else {}
    spec = W.GeometrySpec(kind, "flat", 1, 1, 1, 2.0, 2.0, 2.0, 1, 1, 3.0, 3.0, 1,
                          theta=0.3, sad=100.0, sdd=200.0, **kw)
    g = _gpu(ct, spec)
    for proj in PROJECTORS:
        x = torch.ones((1, 1, 1), device="cuda")
        y = ct.forward(g, x, proj)
        ref = oracle.forward(spec, proj, np.ones((1, 1, 1)))
        assert rel_l2(y.cpu().numpy(), ref) <= TOL_F32
        xb = ct.back(g, torch.ones((1, 1, 1), device="cuda"), proj)
        refb = oracle.back(spec, proj, np.ones((1, 1, 1)))
        assert rel_l2(xb.cpu().numpy(), refb) <= TOL_F32


@pytest.mark.parametrize("kind", ["circ3d", "noncirc3d"])
def test_volume_outside_detector_gives_zero(ct, kind):
    """A detector offset so far that no ray meets the volume: all zeros."""
    kw = dict(phi=[0.05, -0.05, 0.02]) if kind == "noncirc3d" else {}
    spec = W.GeometrySpec(kind, "flat", 8, 8, 8, 1.0, 1.0, 1.0, 16, 16, 1.0, 1.0, 3,
                          theta=[0.0, 1.0, 2.0], sad=200.0, sdd=400.0, u_ofst=500.0, **kw)
    g = _gpu(ct, spec)
    x = torch.ones((8, 8, 8), device="cuda")
    for proj in PROJECTORS:
        assert float(ct.forward(g, x, proj).abs().max()) == 0.0
        assert float(ct.back(g, torch.ones((3, 16, 16), device="cuda"), proj).abs().max()) == 0.0


def _noncirc_regime(regime):
    """Non-circular geometries whose footprints take each kernel variant
    (the ragged geometry itself takes 4 cells x 3 rows):
    'rows4'  -- axial half height in (1, 1.5] rows, two 64-row tiles;
    'cells6' -- transaxial half width in (1.5, 2.5] cells;
    'cells8' -- transaxial half width in (2.5, 3.5] cells;
    'wide'   -- transaxial half width above 3.5 cells (the general kernels)."""
    import dataclasses
    spec = ragged("noncirc3d", "flat", seed=7)
    if regime == "rows4":
        return dataclasses.replace(spec, nv=75, dv=1.1)
    if regime == "cells6":
        return dataclasses.replace(spec, nu=100, du=1.3)
    if regime == "cells8":
        return dataclasses.replace(spec, nu=150, du=0.9)
    return dataclasses.replace(spec, nu=220, du=0.6)


@pytest.mark.parametrize("proj", ["sf", "dd"])
@pytest.mark.parametrize("regime", ["rows4", "cells6", "cells8", "wide"])
def test_noncirc_footprint_regimes(ct, regime, proj):
    spec = _noncirc_regime(regime)
    g = _gpu(ct, spec)
    x = W.phantom(spec, seed=3)
    ref = oracle.forward(spec, proj, x)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).cuda(), proj)
    err = rel_l2(y.cpu().numpy().reshape(ref.shape), ref)
    assert err <= TOL_F32, f"{regime}/{proj} forward: rel L2 {err:.3e}"
    s = W.random_sino(spec, seed=4)[0]
    refb = oracle.back(spec, proj, s)
    xb = ct.back(g, torch.as_tensor(s.reshape(ct_sino_shape(spec)), dtype=torch.float32).cuda(), proj)
    err = rel_l2(xb.cpu().numpy().reshape(refb.shape), refb)
    assert err <= TOL_F32, f"{regime}/{proj} back: rel L2 {err:.3e}"


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_long_object_beyond_the_detector(ct, det):
    """A volume whose z extent projects about 30 rows past both ends of the
    detector (a long object in a circular scan): whole 16-voxel chunks of a
    column fall above or below the detector, voxels 0.8 mm tall project
    shorter than a row (the back kernels' row-filter path).  Every projector,
    both directions, and the recon-mode backprojection."""
    import dataclasses
    spec = dataclasses.replace(ragged("circ3d", det, seed=65), nz=120, dz=0.8)
    g = _gpu(ct, spec)
    x = W.phantom(spec, seed=1)
    s = W.random_sino(spec, seed=2)[0]
    xt = torch.as_tensor(x, dtype=torch.float32).cuda()
    st = torch.as_tensor(s, dtype=torch.float32).cuda()
    for proj in PROJECTORS + (["sftt"] if det == "flat" else []):
        ref = oracle.forward(spec, proj, x)
        assert rel_l2(ct.forward(g, xt, proj).cpu().numpy(), ref) <= TOL_F32, proj
        refb = oracle.back(spec, proj, s)
        assert rel_l2(ct.back(g, st, proj).cpu().numpy(), refb) <= TOL_F32, proj
    q = oracle.ramp_filter(spec, oracle.forward(spec, "dd", x))
    qt = torch.as_tensor(q, dtype=torch.float32).cuda()
    for proj in ("voxel", "dd", "sf"):
        ref = oracle.back_recon(spec, q, proj)
        assert rel_l2(ct.back(g, qt, proj, mode="recon").cpu().numpy(), ref) <= TOL_F32, proj


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_ray_back_narrow_shadows(ct, det):
    """Cells wider than a voxel's shadow (footprint bound below one cell): the
    circular ray back takes its two-cell groups; forward and back against the
    oracle, and the adjoint identity."""
    import dataclasses
    spec = dataclasses.replace(ragged("circ3d", det, seed=67), nu=42, du=3.2)
    g = _gpu(ct, spec)
    x = W.phantom(spec, seed=3)
    s = W.random_sino(spec, seed=4)[0]
    xt = torch.as_tensor(x, dtype=torch.float32).cuda()
    st = torch.as_tensor(s, dtype=torch.float32).cuda()
    y = ct.forward(g, xt, "ray")
    assert rel_l2(y.cpu().numpy(), oracle.forward(spec, "ray", x)) <= TOL_F32
    xb = ct.back(g, st, "ray")
    assert rel_l2(xb.cpu().numpy(), oracle.back(spec, "ray", s)) <= TOL_F32
    lhs = float((y.double() * st.double()).sum())
    rhs = float((xt.double() * xb.double()).sum())
    assert abs(lhs - rhs) <= TOL_F32 * abs(lhs)
