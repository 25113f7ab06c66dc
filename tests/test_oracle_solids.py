"""Pins of the oracle's footprint and voxel-driven projectors against the
exact line integrals of uniform solids (Sec. 2.3; the footprint methods
cited there integrate each voxel's shadow over the detector cell).

* The projection of a voxelised ball (circular cone beam, flat and curved
  detectors) and of a rotated, off-centre ellipsoid (tilted non-circular
  pose with source and detector offsets) converges, as the voxel shrinks
  under a fixed detector, to the exact line integral averaged over each
  detector cell.  The reference
  averages 24 x 24 rays per cell (accurate to ~3e-5 here); each ray's
  chord through the quadric is exact.
* The same in fan beam (flat and curved detectors) for a rotated ellipse,
  the reference averaging each cell's width.
* Footprint mass: the total projected mass of SF-TR, DD and SF-TT equals
  the voxelised object's exact cell-integrated projection (to ~1e-5).
  Under an in-plane detector roll psi it equals cos^2 psi of it.  This is
  the reading of these projectors under roll: the transaxial width is taken
  along e_u and the axial height along e_v, and each is the cos psi-shortened
  extent of a shadow whose area the roll leaves unchanged.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from test_oracle_ray import _rotation

MU = 0.02
NU, NV, DU = 27, 21, 3.0
BALL = (np.array([5.0, -3.0, 4.0]), np.eye(3) / 18.0 ** 2)
_R = _rotation(0.4, -0.7, 0.3)
ELLIPSOID = (np.array([-4.0, 3.0, -2.0]), _R @ np.diag([1 / 20.0 ** 2, 1 / 14.0 ** 2, 1 / 10.0 ** 2]) @ _R.T)
TILTED = dict(theta=2.2, phi=0.15, z_src=3.0, u_ofst=1.5, v_ofst=-2.0)


def _spec(kind, n, det="flat", **kw):
    h = 64.0 / n
    return W.GeometrySpec(kind, det, n, n, n, h, h, h, NU, NV, DU, DU, 1, sad=300.0, sdd=600.0, **kw)


def _voxelise(spec, c, Q):
    g = (np.arange(spec.nx) - (spec.nx - 1) / 2) * spec.dx
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1)
    return np.where(np.einsum("...i,ij,...j->...", P, Q, P) <= 1.0, MU, 0.0)


def _cell_average(spec, c, Q, S=24):
    """mu x the chord of the quadric (X - c)^T Q (X - c) <= 1, averaged over
    S x S rays per detector cell: offsets along e_u and e_v on a flat
    detector; along the arc (angle step du / D about the source's e_v axis)
    and the height on a curved one."""
    f = oracle.frame(spec, 0)
    s = f["s"]
    P = np.array([[oracle.cell_point(spec, 0, a, b) for a in range(spec.nu)] for b in range(spec.nv)])
    o = (np.arange(S) + 0.5) / S - 0.5
    if spec.det == "curved":
        r = P - s
        A = np.arctan2(r @ f["eu"], r @ f["n"])[:, :, None, None] + (o * spec.du / f["D"])[None, None, :, None]
        T = (r @ f["ev"])[:, :, None, None] + (o * spec.dv)[None, None, None, :]
        sub = s + f["D"] * (np.sin(A)[..., None] * f["eu"] + np.cos(A)[..., None] * f["n"]) + T[..., None] * f["ev"]
    else:
        sub = (P[:, :, None, None, :] + (o[:, None] * spec.du * f["eu"])[None, None, :, None, :]
               + (o[:, None] * spec.dv * f["ev"])[None, None, None, :, :])
    d = sub - s
    w = s - c
    alpha = np.einsum("...i,ij,...j->...", d, Q, d)
    beta = np.einsum("...i,ij,j->...", d, Q, w)
    disc = beta * beta - alpha * (w @ Q @ w - 1.0)
    chord = np.where(disc > 0, 2 * np.sqrt(np.maximum(disc, 0.0)) / alpha * np.linalg.norm(d, axis=-1), 0.0)
    return MU * chord.mean(axis=(2, 3))


def _errors(kind, solid, proj, ns, det="flat", **kw):
    c, Q = solid
    ref = _cell_average(_spec(kind, ns[0], det, **kw), c, Q)
    assert (ref > 0).sum() > 100
    errs = []
    for n in ns:
        spec = _spec(kind, n, det, **kw)
        y = oracle.forward(spec, proj, _voxelise(spec, c, Q))[0]
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    return errs


def _converges(errs, final, rate=None):
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    if rate is not None:
        assert all(e0 / e1 > rate for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < final, errs


@pytest.mark.parametrize("proj, det", [("sf", "flat"), ("dd", "flat"), ("sftt", "flat"),
                                       ("sf", "curved"), ("dd", "curved")])
def test_footprint_projection_of_a_ball_converges_to_cell_averaged_integral(proj, det, report):
    errs = _errors("circ3d", BALL, proj, (16, 32, 64, 128), det, theta=0.5)
    report("rel L2 at 16^3 .. 128^3: " + ", ".join(f"{e:.2e}" for e in errs))
    _converges(errs, 0.006, rate=1.6)


@pytest.mark.parametrize("proj", ["sf", "dd", "sftt"])
def test_footprint_projection_of_an_ellipsoid_converges_noncircular(proj, report):
    errs = _errors("noncirc3d", ELLIPSOID, proj, (16, 32, 64, 128), **TILTED)
    report("rel L2 at 16^3 .. 128^3: " + ", ".join(f"{e:.2e}" for e in errs))
    _converges(errs, 0.01, rate=1.6)


@pytest.mark.parametrize("kind, det, solid, kw", [("circ3d", "flat", BALL, dict(theta=0.5)),
                                                  ("circ3d", "curved", BALL, dict(theta=0.5)),
                                                  ("noncirc3d", "flat", ELLIPSOID, TILTED)])
def test_voxel_driven_projection_converges_to_cell_averaged_integral(kind, det, solid, kw):
    _converges(_errors(kind, solid, "voxel", (32, 64, 128), det, **kw), 0.02)


def test_ray_driven_projection_samples_the_cell_centre():
    """The ray-driven projection samples each cell's centre: against the cell
    average it stalls at the averaging's own size (~2.5 % here) while the
    footprint methods go below 0.5 %, so the cell-average pins above tell
    the two kinds of detector model apart."""
    errs = _errors("circ3d", BALL, "ray", (32, 64, 128), "curved", theta=0.5)
    assert errs[-1] > 0.015 and errs[-1] / errs[-2] > 0.7, errs


def _fan_errors(proj, det, ns):
    """Fan beam: a rotated, off-centre uniform ellipse (semi-axes 22 and 12
    mm) against its exact chord averaged over each cell's width (64 rays per
    cell, along the line or the arc)."""
    c = np.array([6.0, -4.0, 0.0])
    R = _rotation(0.6, 0.0, 0.0)
    Q = R @ np.diag([1 / 22.0 ** 2, 1 / 12.0 ** 2, 0.0]) @ R.T

    def spec_(n):
        h = 64.0 / n
        return W.GeometrySpec("fan2d", det, n, n, 1, h, h, 1.0, 61, 1, 1.6, 1.0, 1, theta=1.1, sad=400.0, sdd=800.0)

    spec = spec_(ns[0])
    f = oracle.frame(spec, 0)
    s = f["s"]
    P = np.array([oracle.cell_point(spec, 0, a, 0) for a in range(spec.nu)])
    o = (np.arange(64) + 0.5) / 64 - 0.5
    if det == "curved":
        r = P - s
        A = np.arctan2(r @ f["eu"], r @ f["n"])[:, None] + o[None, :] * spec.du / f["D"]
        sub = s + f["D"] * (np.sin(A)[..., None] * f["eu"] + np.cos(A)[..., None] * f["n"]) \
            + (r @ f["ev"])[:, None, None] * f["ev"]
    else:
        sub = P[:, None, :] + (o[:, None] * spec.du * f["eu"])[None, :, :]
    d = sub - s
    w = s - c
    alpha = np.einsum("...i,ij,...j->...", d, Q, d)
    beta = np.einsum("...i,ij,j->...", d, Q, w)
    disc = beta * beta - alpha * (w @ Q @ w - 1.0)
    ref = MU * np.where(disc > 0, 2 * np.sqrt(np.maximum(disc, 0.0)) / alpha * np.linalg.norm(d, axis=-1), 0.0).mean(1)
    assert (ref > 0).sum() > 20
    errs = []
    for n in ns:
        spec = spec_(n)
        g = (np.arange(n) - (n - 1) / 2) * spec.dx
        X, Y = np.meshgrid(g, g)
        Pp = np.stack([X - c[0], Y - c[1], np.zeros_like(X)], axis=-1)
        img = np.where(np.einsum("...i,ij,...j->...", Pp, Q, Pp) <= 1.0, MU, 0.0)[None]
        y = oracle.forward(spec, proj, img)[0, 0]
        errs.append(np.linalg.norm(y - ref) / np.linalg.norm(ref))
    return errs


@pytest.mark.parametrize("det", ["flat", "curved"])
@pytest.mark.parametrize("proj", ["sf", "dd", "voxel"])
def test_fan_beam_projection_of_an_ellipse_converges_to_cell_averaged_integral(proj, det, report):
    errs = _fan_errors(proj, det, (32, 64, 128, 256))
    report("rel L2 at 32^2 .. 256^2: " + ", ".join(f"{e:.2e}" for e in errs))
    _converges(errs, 0.005, rate=1.6)


@pytest.mark.parametrize("proj", ["sf", "dd", "sftt"])
@pytest.mark.parametrize("psi", [0.0, 0.1, 0.3])
def test_footprint_mass_and_detector_roll(proj, psi, report):
    """Total projected mass / the voxelised ball's exact cell-integrated
    projection: 1 without roll (mass conservation), cos^2 psi under a roll."""
    r = 8.0
    c, Q = np.zeros(3), np.eye(3) / r ** 2
    spec = _spec("noncirc3d", 64, theta=2.2, psi=psi)
    x = _voxelise(spec, c, Q)
    vol = x.sum() / MU * spec.dx ** 3 / (4.0 / 3.0 * math.pi * r ** 3)  # voxelised / exact volume
    ratio = oracle.forward(spec, proj, x)[0].sum() / _cell_average(spec, c, Q).sum() / vol
    report(f"mass ratio {ratio:.6f}, cos^2 psi {math.cos(psi) ** 2:.6f}")
    assert abs(ratio - math.cos(psi) ** 2) < 2e-4, (ratio, math.cos(psi) ** 2)


@pytest.mark.parametrize("psi", [0.0, 0.1, 0.3])
def test_voxel_driven_mass_is_exact_under_roll(psi, report):
    """The voxel-driven projection spreads each voxel's exact projected mass
    (R8's amplitude) over bilinear weights that sum to one, so its total
    equals the voxelised ball's exact cell-integrated projection at any
    roll; the cos^2 psi of the footprint methods is theirs alone."""
    r = 8.0
    c, Q = np.zeros(3), np.eye(3) / r ** 2
    spec = _spec("noncirc3d", 64, theta=2.2, psi=psi)
    x = _voxelise(spec, c, Q)
    vol = x.sum() / MU * spec.dx ** 3 / (4.0 / 3.0 * math.pi * r ** 3)
    ratio = oracle.forward(spec, "voxel", x)[0].sum() / _cell_average(spec, c, Q).sum() / vol
    report(f"mass ratio {ratio:.7f}")
    assert abs(ratio - 1.0) < 2e-5, ratio
