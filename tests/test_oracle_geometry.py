"""Pins of the oracle's geometry (Sec. 2.2, Table 1) against hand-derived
frames and projections stored under tests/golden/."""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            yield line


def test_frames_match_hand_derivation():
    for line in _rows("frames.txt"):
        head, s, c, eu, ev = [p.split() for p in line.split("|")]
        th, ph, ps, sad, sdd, xs, zs, uo, vo = map(float, head)
        d2r = math.pi / 180
        spec = W.GeometrySpec("noncirc3d", "flat", 4, 4, 4, 1, 1, 1, 4, 4, 1, 1, 1,
                              theta=th * d2r, phi=ph * d2r, psi=ps * d2r, sad=sad, sdd=sdd,
                              x_src=xs, z_src=zs, u_ofst=uo, v_ofst=vo)
        f = oracle.frame(spec, 0)
        for key, want in (("s", s), ("c", c), ("eu", eu), ("ev", ev)):
            np.testing.assert_allclose(f[key], np.array(want, float), atol=1e-9, err_msg=f"{key}: {line}")
        # n = e_u x e_v is the unit detector normal pointing away from the source
        np.testing.assert_allclose(f["n"], np.cross(f["eu"], f["ev"]), atol=1e-12)
        assert f["D"] == pytest.approx(sdd, abs=1e-9)


def test_projection_matches_hand_derivation():
    for line in _rows("projections.txt"):
        det, x, y, z, u, v = line.split()
        spec = W.GeometrySpec("circ3d", det, 4, 4, 4, 1, 1, 1, 4, 4, 1, 1, 1,
                              theta=0.0, sad=500.0, sdd=1000.0)
        uv = oracle.project(spec, 0, [float(x), float(y), float(z)])
        np.testing.assert_allclose(uv, [float(u), float(v)], rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_cell_points_project_back_to_cell_centres(det):
    spec = W.GeometrySpec("circ3d", det, 4, 4, 4, 1, 1, 1, 9, 5, 3.0, 2.5, 3,
                          theta=[0.3, 1.9, -2.2], sad=600.0, sdd=1100.0,
                          x_src=1.5, z_src=-2.0, u_ofst=4.0, v_ofst=-3.0)
    for v in range(3):
        f = oracle.frame(spec, v)
        for a in (0, 4, 8):
            for b in (0, 2, 4):
                P = oracle.cell_point(spec, v, a, b)
                uv = oracle.project(spec, v, f["s"] + 0.6 * (P - f["s"]))
                np.testing.assert_allclose(uv, [(a - 4) * 3.0, (b - 2) * 2.5], atol=1e-9)


def test_curved_cells_lie_on_the_source_cylinder():
    spec = W.GeometrySpec("circ3d", "curved", 4, 4, 4, 1, 1, 1, 11, 3, 20.0, 4.0, 1,
                          theta=0.7, sad=600.0, sdd=1100.0, u_ofst=7.0)
    f = oracle.frame(spec, 0)
    for a in range(11):
        P = oracle.cell_point(spec, 0, a, 1)
        w = P - f["s"]
        rho = math.hypot(w @ f["eu"], w @ f["n"])
        assert rho == pytest.approx(1100.0, rel=1e-13)
    # neighbouring cells are one arc length du apart on the circle of radius SDD
    P0 = oracle.cell_point(spec, 0, 3, 1) - f["s"]
    P1 = oracle.cell_point(spec, 0, 4, 1) - f["s"]
    ang = math.acos(P0 @ P1 / (np.linalg.norm(P0) * np.linalg.norm(P1)))
    assert ang * 1100.0 == pytest.approx(20.0, rel=1e-10)


def test_noncircular_with_zero_tilts_equals_circular():
    """Sec. 2.2: the non-circular geometry with phi = psi = 0 is the circular one."""
    circ = W.scaled(W.circ3d_256(), 12, 7)
    circ.x_src, circ.z_src, circ.u_ofst, circ.v_ofst = 1.0, -2.0, 3.0, 0.5
    nonc = W.GeometrySpec(**{**circ.__dict__, "kind": "noncirc3d"})
    x = W.random_volume(circ, 3)[0]
    for p in ("voxel", "ray", "dd", "sf"):
        np.testing.assert_array_equal(oracle.forward(circ, p, x), oracle.forward(nonc, p, x))


def test_poses_reproduce_angle_parametrisation():
    spec = W.scaled(W.noncirc3d_saddle(), 10, 5)
    poses = []
    for v in range(spec.nview):
        f = oracle.frame(spec, v)
        poses.append(np.concatenate([f["s"], f["c"], f["eu"], f["ev"]]))
    posed = W.GeometrySpec(**{**spec.__dict__, "poses": np.array(poses)})
    x = W.random_volume(spec, 1)[0]
    for p in ("voxel", "ray", "dd", "sf"):
        np.testing.assert_allclose(oracle.forward(posed, p, x), oracle.forward(spec, p, x),
                                   rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("proj", ["ray", "dd", "sf"])
def test_single_slice_3d_equals_2d(proj):
    """Sec. 2.2: a 3D geometry with a single slice reduces to the 2D one.  With
    unit slice thickness and unit row height the slice covers its row."""
    fan = W.GeometrySpec("fan2d", "flat", 20, 16, 1, 2.0, 2.0, 1.0, 40, 1, 2.5, 1.0, 9,
                         theta=np.linspace(0, 5, 9), sad=300.0, sdd=600.0, x_src=1.0,
                         u_ofst=2.0, x_ofst=3.0, y_ofst=-1.0)
    cone = W.GeometrySpec(**{**fan.__dict__, "kind": "circ3d"})
    x = W.random_volume(fan, 0)[0]
    np.testing.assert_allclose(oracle.forward(cone, proj, x), oracle.forward(fan, proj, x),
                               rtol=1e-12, atol=1e-13)
