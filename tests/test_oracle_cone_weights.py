"""Cone-beam pins of the oracle's SF-TR, DD and SF-TT weights (Sec. 2.3: the
separable footprint of Long, Fessler & Balter 2010 and the distance-driven
projector of De Man & Basu 2004).

The parallel-limit and fan-beam pins elsewhere see rays with no z component,
so they cannot tell the 3D ray length from its transaxial part.  Here every
case has rays well off the mid-plane:

* hand-derived weights of one voxel off the mid-plane (`golden/cone_weights.txt`,
  derivation in its header), flat and curved detectors;
* the 3D mass identities on circular flat, circular curved and non-circular
  geometries, with the amplitudes and path lengths measured as chords of
  rays through boxes by the brute-force slab method (`brute.seg_lengths`),
  not from the oracle's expressions.
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from brute import seg_lengths

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cone_weights.txt")
BIG = 1.0e6  # half-extent of an "infinite" box side (mm)


def _golden_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            det, proj, a, b, rest = line.split(None, 4)
            expr, value = rest.rsplit(None, 1)
            rows.append((det, proj, int(a), int(b), expr, float(value)))
    return rows


def _golden_spec(det):
    return W.GeometrySpec("circ3d", det, 21, 21, 61, 2.0, 2.0, 2.0, 64, 64, 8.0, 4.0, 1,
                          theta=0.0, sad=500.0, sdd=1000.0)


ROWS = _golden_rows()


@pytest.mark.parametrize("row", ROWS, ids=[f"{r[0]}-{r[1]}-{r[2]}-{r[3]}" for r in ROWS])
def test_off_midplane_voxel_matches_hand_derived_weights(row):
    det, proj, a, b, expr, value = row
    ns = {"sqrt": math.sqrt, "atan2": math.atan2, "cos": math.cos, "__builtins__": {}}
    want = eval(expr, ns)  # noqa: S307 -- the golden file's own arithmetic
    assert want == pytest.approx(value, rel=1e-14)
    aa, bb, w = oracle.footprint(_golden_spec(det), proj, 0, 15, 12, 60)
    got = {(int(x), int(y)): float(z) for x, y, z in zip(aa, bb, w)}
    assert set(got) == {(34, 61), (34, 62)}
    assert got[(a, b)] == pytest.approx(want, rel=1e-13)


def test_golden_cases_are_off_the_midplane():
    """The 3D factors of the golden voxel differ from their transaxial parts
    by more than 0.5 %, far above the 1e-13 the test holds the weights to."""
    w = np.array([10.0, -496.0, 60.0])
    assert np.linalg.norm(w) / np.linalg.norm(w[:2]) > 1.005
    d = np.array([20.0, -1000.0, 118.0])
    assert np.linalg.norm(d) / np.linalg.norm(d[:2]) > 1.005


# ---------------------------------------------------------------- 3D mass identities

CONE_CASES = [
    W.GeometrySpec("circ3d", "flat", 9, 9, 9, 1.0, 1.0, 1.3, 48, 48, 0.9, 0.8, 3,
                   theta=[0.2, 1.1, 2.6], sad=50.0, sdd=110.0, x_src=1.5, z_src=-2.0,
                   u_ofst=0.7, v_ofst=-1.1),
    W.GeometrySpec("circ3d", "curved", 9, 9, 9, 1.0, 1.0, 1.3, 48, 48, 0.9, 0.8, 3,
                   theta=[0.2, 1.1, 2.6], sad=50.0, sdd=110.0, x_src=1.5, z_src=-2.0,
                   u_ofst=0.7, v_ofst=-1.1),
    W.GeometrySpec("noncirc3d", "flat", 9, 9, 9, 1.0, 1.0, 1.3, 48, 48, 0.9, 0.8, 3,
                   theta=[0.2, 1.1, 2.6], phi=[0.15, -0.2, 0.05], psi=[0.03, 0.0, -0.1],
                   sad=50.0, sdd=110.0, z_src=[3.0, -2.0, 0.0], u_ofst=0.7),
]
CONE_IDS = ["circ-flat", "circ-curved", "noncirc"]
# voxels away from the mid-plane (k far from 4) and off the axis
VOXELS = [(0, 0, 0), (8, 3, 8), (2, 7, 1), (5, 5, 7)]


def _centre(spec, i, j, k):
    return np.array([(i - 0.5 * (spec.nx - 1)) * spec.dx, (j - 0.5 * (spec.ny - 1)) * spec.dy,
                     (k - 0.5 * (spec.nz - 1)) * spec.dz])


def _column_chord(s, X, h):
    """3D length of the line from s through X inside the infinite square
    column |x - X_x| <= h, |y - X_y| <= h (any z)."""
    P = s + 4.0 * (X - s)
    lo = np.array([[X[0] - h, X[1] - h, -BIG]])
    hi = np.array([[X[0] + h, X[1] + h, BIG]])
    return float(seg_lengths(s, P, lo, hi)[0])


def _slab_chord(s, P, axis, centre, width):
    """3D length of the segment s -> P inside the slab |X_axis - centre| <= width/2."""
    lo = np.full((1, 3), -BIG)
    hi = np.full((1, 3), BIG)
    lo[0, axis] = centre - 0.5 * width
    hi[0, axis] = centre + 0.5 * width
    return float(seg_lengths(s, P, lo, hi)[0])


@pytest.mark.parametrize("spec", CONE_CASES, ids=CONE_IDS)
@pytest.mark.parametrize("voxel", VOXELS)
@pytest.mark.parametrize("view", [0, 1, 2])
def test_sf_cone_mass_identity(spec, voxel, view):
    """sum_c w du dv = A1 * area_u * (v+ - v-): the trapezoid's area from the
    four projected column corners, the rectangle's height from the projected
    end points, and A1 the chord of the central ray through the voxel's
    infinite square column (Long et al.'s amplitude), measured by the slab
    method."""
    i, j, k = voxel
    f = oracle.frame(spec, view)
    X = _centre(spec, i, j, k)
    t = sorted(oracle.project(spec, view, X + [sx * 0.5, sy * 0.5, 0.0])[0]
               for sx in (-1.0, 1.0) for sy in (-1.0, 1.0))
    area = 0.5 * (t[3] + t[2] - t[1] - t[0])
    v1 = oracle.project(spec, view, X - [0.0, 0.0, 0.5 * spec.dz])[1]
    v2 = oracle.project(spec, view, X + [0.0, 0.0, 0.5 * spec.dz])[1]
    a1 = _column_chord(np.asarray(f["s"]), X, 0.5 * spec.dx)
    _, _, w = oracle.footprint(spec, "sf", view, i, j, k)
    assert w.sum() * spec.du * spec.dv == pytest.approx(a1 * area * abs(v2 - v1), rel=1e-12)


@pytest.mark.parametrize("spec", CONE_CASES, ids=CONE_IDS)
@pytest.mark.parametrize("voxel", VOXELS)
@pytest.mark.parametrize("view", [0, 1, 2])
def test_dd_cone_partition_identity(spec, voxel, view):
    """With each cell's path length L_c divided out, the DD weights of an
    interior voxel sum to (u+ - u-)(v+ - v-) / (du dv).  L_c is measured as
    the 3D chord of the cell's ray through one slab of the main axis (the
    slab around the voxel), by the slab method."""
    i, j, k = voxel
    f = oracle.frame(spec, view)
    s = np.asarray(f["s"])
    X = _centre(spec, i, j, k)
    cs = np.asarray(f["c"]) - s
    my = abs(cs[1]) >= abs(cs[0])  # main axis (R10): y unless x dominates
    off = np.array([0.5 * spec.dx, 0.0, 0.0]) if my else np.array([0.0, 0.5 * spec.dy, 0.0])
    u1 = oracle.project(spec, view, X - off)[0]
    u2 = oracle.project(spec, view, X + off)[0]
    v1 = oracle.project(spec, view, X - [0.0, 0.0, 0.5 * spec.dz])[1]
    v2 = oracle.project(spec, view, X + [0.0, 0.0, 0.5 * spec.dz])[1]
    a, b, w = oracle.footprint(spec, "dd", view, i, j, k)
    axis = 1 if my else 0
    width = spec.dy if my else spec.dx
    tot = 0.0
    for aa, bb, ww in zip(a, b, w):
        P = oracle.cell_point(spec, view, int(aa), int(bb))
        tot += ww / _slab_chord(s, P, axis, X[axis], width)
    want = abs(u2 - u1) * abs(v2 - v1) / (spec.du * spec.dv)
    assert tot == pytest.approx(want, rel=1e-12)
