"""Pins of the oracle's SF-TT weights (Long, Fessler & Balter 2010, cited in
Sec. 2.3; the trapezoid-trapezoid variant with the per-cell amplitude A2):
with the amplitude of each cell divided out, a voxel's weights sum to the
product of its two trapezoid areas -- the transaxial one from the four
column corners, the axial one from the z faces at the corners nearest to
and farthest from the source -- recomputed here from the pinned detector
mapping, not from the footprint code; A2 itself is measured as a chord by the
slab method.  Hand-derived SF-TT weights off the mid-plane are pinned in
test_oracle_cone_weights.py."""
import numpy as np
import pytest

import oracle
import workloads as W
from brute import seg_lengths


def _expected(spec, view, i, j, k):
    f = oracle.frame(spec, view)
    X = np.array([(i - 0.5 * (spec.nx - 1)) * spec.dx, (j - 0.5 * (spec.ny - 1)) * spec.dy,
                  0.0 if spec.kind == "fan2d" else (k - 0.5 * (spec.nz - 1)) * spec.dz])
    dz = 1.0 if spec.kind == "fan2d" else spec.dz
    dv = 1.0 if spec.kind == "fan2d" else spec.dv
    corners = [(sx, sy) for sx in (-1, 1) for sy in (-1, 1)]
    tau, depth = [], []
    for sx, sy in corners:
        P = X + np.array([0.5 * sx * spec.dx, 0.5 * sy * spec.dy, 0.0])
        tau.append(oracle.project(spec, view, P)[0])
        depth.append(float((P - f["s"]) @ f["n"]))
    tau = np.sort(tau)
    tv = []
    for c in (int(np.argmin(depth)), int(np.argmax(depth))):
        sx, sy = corners[c]
        for sz in (-1, 1):
            P = X + np.array([0.5 * sx * spec.dx, 0.5 * sy * spec.dy, 0.5 * sz * dz])
            tv.append(oracle.project(spec, view, P)[1])
    tv = np.sort(tv)
    area_u = 0.5 * (tau[3] + tau[2] - tau[1] - tau[0])
    if spec.kind == "fan2d":
        # a single row of unit height inside the axial plateau (magnification
        # > 1): the axial factor is 1 and the weights are the line integrals'
        assert tv[1] < -0.5 and tv[2] > 0.5
        return area_u / spec.du, f
    area_v = 0.5 * (tv[3] + tv[2] - tv[1] - tv[0])
    return area_u / spec.du * area_v / dv, f


def _a2(spec, f, view, a, b):
    """A2 measured, not recomputed: the 3D chord of the ray from the source
    to the cell centre through a square column of side dx centred on that
    ray (Long et al.'s amplitude taken along the cell's ray), found by the
    brute-force slab method."""
    s = np.asarray(f["s"])
    C = oracle.cell_point(spec, view, int(a), int(b))
    M = 0.5 * (s + C)
    h = 0.5 * spec.dx
    lo = np.array([[M[0] - h, M[1] - h, -1.0e6]])
    hi = np.array([[M[0] + h, M[1] + h, 1.0e6]])
    return float(seg_lengths(s, s + 4.0 * (C - s), lo, hi)[0])


CASES = [
    W.GeometrySpec("circ3d", "flat", 9, 9, 9, 1.0, 1.0, 1.3, 40, 40, 1.0, 1.0, 3,
                   theta=[0.2, 1.1, 2.6], sad=60.0, sdd=120.0),
    W.GeometrySpec("circ3d", "curved", 9, 9, 9, 1.0, 1.0, 1.3, 40, 40, 1.0, 1.0, 3,
                   theta=[0.2, 1.1, 2.6], sad=60.0, sdd=120.0),
    W.GeometrySpec("noncirc3d", "flat", 9, 9, 9, 1.0, 1.0, 1.3, 40, 40, 1.0, 1.0, 3,
                   theta=[0.2, 1.1, 2.6], phi=[0.1, -0.2, 0.05], psi=[0.03, 0.0, -0.1],
                   sad=60.0, sdd=120.0, z_src=[3.0, -2.0, 0.0]),
    W.GeometrySpec("fan2d", "flat", 9, 9, 1, 1.0, 1.0, 1.0, 40, 1, 1.0, 1.0, 3,
                   theta=[0.2, 1.1, 2.6], sad=60.0, sdd=120.0),
]


@pytest.mark.parametrize("spec", CASES, ids=["circ-flat", "circ-curved", "noncirc", "fan"])
@pytest.mark.parametrize("voxel", [(0, 0, 0), (4, 4, 4), (8, 3, 6), (2, 7, 1)])
@pytest.mark.parametrize("view", [0, 1, 2])
def test_sftt_weights_sum_to_the_two_trapezoid_areas(spec, voxel, view):
    i, j, k = voxel
    if spec.kind == "fan2d":
        k = 0
    a, b, w = oracle.footprint(spec, "sftt", view, i, j, k)
    want, f = _expected(spec, view, i, j, k)
    got = sum(wi / _a2(spec, f, view, ai, bi) for ai, bi, wi in zip(a, b, w))
    assert abs(got - want) <= 1e-12 * want


def test_sftt_is_the_exact_adjoint_pair():
    spec = CASES[2]
    rng = np.random.default_rng(0)
    x = rng.random(spec.vol_shape)
    y = rng.random(spec.sino_shape)
    lhs = float((oracle.forward(spec, "sftt", x) * y).sum())
    rhs = float((x * oracle.back(spec, "sftt", y)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
