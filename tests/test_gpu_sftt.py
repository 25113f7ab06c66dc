"""SF-TT (trapezoid x trapezoid, per-cell amplitude A2; Long, Fessler &
Balter 2010, cited in Sec. 2.3) on the GPU against the FP64 oracle, on the
flat-detector geometries it is provided for."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import TOL_F16, TOL_F32, ragged, rel_l2

pytestmark = pytest.mark.gpu

FLAT = [("fan2d", "flat"), ("circ3d", "flat"), ("noncirc3d", "flat")]


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _vol(spec):
    return (spec.ny, spec.nx) if spec.kind == "fan2d" else spec.vol_shape


def _sino(spec):
    return (spec.nview, spec.nu) if spec.kind == "fan2d" else spec.sino_shape


@pytest.mark.parametrize("kind,det", FLAT)
def test_sftt_forward_and_back_match_oracle(ct, kind, det):
    spec = ragged(kind, det, seed=60)
    g = ct.Geometry.from_spec(spec)
    x = W.phantom(spec, seed=1)
    ref = oracle.forward(spec, "sftt", x)
    y = ct.forward(g, torch.as_tensor(x.reshape(_vol(spec)), dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(y.cpu().numpy().reshape(ref.shape), ref) <= TOL_F32
    s = W.random_sino(spec, seed=2)[0]
    refb = oracle.back(spec, "sftt", s)
    xb = ct.back(g, torch.as_tensor(s.reshape(_sino(spec)), dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(xb.cpu().numpy().reshape(refb.shape), refb) <= TOL_F32


@pytest.mark.parametrize("regime", ["rows4", "cells8"])
def test_sftt_footprint_regimes(ct, regime):
    spec = ragged("noncirc3d", "flat", seed=61)
    # rows4: the axial trapezoid's bound in (1, 1.5] rows (about 1.28), two 64-row tiles
    spec = (dataclasses.replace(spec, nv=70, dv=1.4) if regime == "rows4"
            else dataclasses.replace(spec, nu=150, du=0.9))
    g = ct.Geometry.from_spec(spec)
    x = W.phantom(spec, seed=3)
    ref = oracle.forward(spec, "sftt", x)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(y.cpu().numpy(), ref) <= TOL_F32
    s = W.random_sino(spec, seed=4)[0]
    refb = oracle.back(spec, "sftt", s)
    xb = ct.back(g, torch.as_tensor(s, dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(xb.cpu().numpy(), refb) <= TOL_F32


def test_sftt_adjoint_identity_and_batches(ct):
    spec = ragged("noncirc3d", "flat", seed=62)
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(7)
    x = torch.rand((2,) + spec.vol_shape, generator=gen, device="cuda")
    y = torch.rand((2,) + spec.sino_shape, generator=gen, device="cuda")
    Ax, Aty = ct.forward(g, x, "sftt"), ct.back(g, y, "sftt")
    lhs, rhs = float((Ax.double() * y.double()).sum()), float((x.double() * Aty.double()).sum())
    assert abs(lhs - rhs) <= TOL_F32 * abs(lhs)
    assert torch.equal(Ax[1], ct.forward(g, x[1].contiguous(), "sftt"))
    assert torch.equal(Aty[0], ct.back(g, y[0].contiguous(), "sftt"))


def test_sftt_refuses_what_it_does_not_provide(ct):
    curved = ct.Geometry.from_spec(ragged("circ3d", "curved", seed=63))
    with pytest.raises(ct.CTError):
        ct.forward(curved, torch.rand(curved.vol_shape, device="cuda"), "sftt")
    wide = dataclasses.replace(ragged("noncirc3d", "flat", seed=63), nu=220, du=0.6)
    gw = ct.Geometry.from_spec(wide)
    with pytest.raises(ct.CTError):
        ct.forward(gw, torch.rand(gw.vol_shape, device="cuda"), "sftt")


# circular flat 3D geometry runs the column-walk kernels (transaxial footprint
# once per column and view): the ragged case (strided column reads, one-row
# tiles, voxels taller than a row) plus these regimes
CIRC_REGIMES = {
    # z-major column copy (nz a multiple of 4), 64-row tiles, voxels shorter than a row
    "zmajor": dict(nz=24, nv=70, dz=0.8),
    # transaxial footprints of 5..8 cells
    "cells8": dict(nu=150, du=0.9),
    # axial trapezoids of up to 4 rows, two 64-row tiles
    "rows4": dict(nv=70, dv=1.4),
    # voxels shorter than a row with 64-row tiles and strided column reads
    "short": dict(nz=37, nv=66, dz=0.7),
}


@pytest.mark.parametrize("regime", sorted(CIRC_REGIMES))
def test_sftt_circular_regimes(ct, regime):
    spec = dataclasses.replace(ragged("circ3d", "flat", seed=64), **CIRC_REGIMES[regime])
    g = ct.Geometry.from_spec(spec)
    x = W.phantom(spec, seed=5)
    ref = oracle.forward(spec, "sftt", x)
    y = ct.forward(g, torch.as_tensor(x, dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(y.cpu().numpy(), ref) <= TOL_F32
    s = W.random_sino(spec, seed=6)[0]
    refb = oracle.back(spec, "sftt", s)
    xb = ct.back(g, torch.as_tensor(s, dtype=torch.float32).cuda(), "sftt")
    assert rel_l2(xb.cpu().numpy(), refb) <= TOL_F32


def test_sftt_circular_adjoint_batches_and_half(ct):
    spec = dataclasses.replace(ragged("circ3d", "flat", seed=66), nz=24, nv=70, dz=0.8)
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(8)
    x = torch.rand((2,) + spec.vol_shape, generator=gen, device="cuda")
    y = torch.rand((2,) + spec.sino_shape, generator=gen, device="cuda")
    Ax, Aty = ct.forward(g, x, "sftt"), ct.back(g, y, "sftt")
    lhs, rhs = float((Ax.double() * y.double()).sum()), float((x.double() * Aty.double()).sum())
    assert abs(lhs - rhs) <= TOL_F32 * abs(lhs)
    assert torch.equal(Ax[1], ct.forward(g, x[1].contiguous(), "sftt"))
    assert torch.equal(Aty[0], ct.back(g, y[0].contiguous(), "sftt"))
    # FP16 storage: FP32 arithmetic on the rounded input, one rounding at the store
    xh = x[0].half()
    ref = oracle.forward(spec, "sftt", xh.float().cpu().numpy().astype(np.float64))
    yh = ct.forward(g, xh, "sftt", out_dtype=torch.float16)
    assert rel_l2(yh.float().cpu().numpy(), ref) <= TOL_F16
