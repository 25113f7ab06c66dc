"""Pins of the oracle's ray-driven projector (Siddon 1985, Sec. 2.3).

* all-pairs brute force (slab method per ray and voxel, no traversal);
* closed-form chords through the volume box and through grid-aligned blocks;
* convergence of a voxelised disk to the analytic chord 2 mu sqrt(r^2 - d^2);
* first-order convergence of a voxelised ellipse (fan beam), ball (circular
  cone beam) and rotated ellipsoid (tilted non-circular pose) to the chord
  of the ray line through the quadric.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from brute import ray_system_matrix

TINY = {
    "fan2d-flat": W.GeometrySpec("fan2d", "flat", 7, 6, 1, 3.0, 2.5, 1.0, 13, 1, 2.7, 1.0, 6,
                                 theta=np.linspace(0.1, 6.0, 6), sad=80.0, sdd=150.0,
                                 x_src=1.3, u_ofst=-2.1, x_ofst=0.7, y_ofst=-0.4),
    "fan2d-curved": W.GeometrySpec("fan2d", "curved", 7, 6, 1, 3.0, 2.5, 1.0, 13, 1, 2.7, 1.0, 6,
                                   theta=np.linspace(0.2, 6.1, 6), sad=80.0, sdd=150.0,
                                   u_ofst=3.4, x_ofst=-0.6),
    "circ3d-flat": W.GeometrySpec("circ3d", "flat", 5, 6, 4, 3.0, 3.0, 2.0, 9, 7, 3.1, 2.3, 4,
                                  theta=[0.3, 1.4, 2.9, 4.4], sad=90.0, sdd=160.0,
                                  x_src=0.8, z_src=-1.1, u_ofst=1.7, v_ofst=-0.9, z_ofst=0.5),
    "circ3d-curved": W.GeometrySpec("circ3d", "curved", 5, 6, 4, 3.0, 3.0, 2.0, 9, 7, 3.1, 2.3, 4,
                                    theta=[0.3, 1.4, 2.9, 4.4], sad=90.0, sdd=160.0,
                                    z_src=1.1, u_ofst=-1.7, v_ofst=0.9),
    "noncirc3d": W.GeometrySpec("noncirc3d", "flat", 5, 6, 4, 3.0, 3.0, 2.0, 9, 7, 3.1, 2.3, 4,
                                theta=[0.3, 1.4, 2.9, 4.4], phi=[0.1, -0.2, 0.05, 0.3],
                                psi=[0.02, -0.1, 0.2, 0.0], sad=90.0, sdd=160.0,
                                x_src=[0.5, -0.5, 1.0, 0.0], z_src=1.1, u_ofst=-1.7, v_ofst=0.9),
}


@pytest.mark.parametrize("name", sorted(TINY))
def test_siddon_matches_all_pairs_brute_force(name):
    spec = TINY[name]
    A = ray_system_matrix(spec)
    assert (A > 0).sum() > 50  # the rays do cross the volume
    x = W.random_volume(spec, 4)[0]
    y = W.random_sino(spec, 4)[0]
    fwd = oracle.forward(spec, "ray", x).ravel()
    back = oracle.back(spec, "ray", y).ravel()
    np.testing.assert_allclose(fwd, A @ x.ravel(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(back, A.T @ y.ravel(), rtol=1e-12, atol=1e-12)


def test_ones_volume_gives_box_chord_2d():
    """theta = 0, the ray from (0, SAD) to (u, SAD - SDD) crosses the whole
    square through its top and bottom faces: chord = L sqrt(1 + (u/SDD)^2)."""
    L = 64.0
    spec = W.GeometrySpec("fan2d", "flat", 32, 32, 1, 2.0, 2.0, 1.0, 41, 1, 1.5, 1.0, 1,
                          theta=0.0, sad=400.0, sdd=900.0)
    y = oracle.forward(spec, "ray", np.ones((1, 32, 32)))[0, 0]
    u = (np.arange(41) - 20) * 1.5
    x_top = u * (400 - L / 2) / 900
    x_bot = u * (400 + L / 2) / 900
    full = (np.abs(x_top) < L / 2) & (np.abs(x_bot) < L / 2)
    assert full.sum() > 30
    np.testing.assert_allclose(y[full], (L * np.sqrt(1 + (u / 900) ** 2))[full], rtol=1e-13)


def test_ones_volume_gives_box_chord_3d():
    L = 40.0
    spec = W.GeometrySpec("circ3d", "flat", 20, 20, 20, 2.0, 2.0, 2.0, 15, 11, 2.0, 2.0, 1,
                          theta=0.0, sad=300.0, sdd=700.0)
    y = oracle.forward(spec, "ray", np.ones((20, 20, 20)))[0]
    u = (np.arange(15) - 7) * 2.0
    v = (np.arange(11) - 5) * 2.0
    V, U = np.meshgrid(v, u, indexing="ij")
    want = L * np.sqrt(1 + (U ** 2 + V ** 2) / 700 ** 2)
    ok = np.maximum(np.abs(U), np.abs(V)) * (300 + L / 2) / 700 < L / 2
    np.testing.assert_allclose(y[ok], want[ok], rtol=1e-13)


def test_grid_aligned_block_gives_value_times_chord():
    """A block of voxels j in [8, 20), i in [10, 22) with value mu: a ray that
    enters and leaves through the block's y faces has chord 12 dy sqrt(1+t^2)."""
    mu = 0.017
    img = np.zeros((1, 32, 32))
    img[0, 8:20, 10:22] = mu
    spec = W.GeometrySpec("fan2d", "flat", 32, 32, 1, 1.0, 1.0, 1.0, 64, 1, 0.5, 1.0, 1,
                          theta=0.0, sad=500.0, sdd=1000.0)
    y = oracle.forward(spec, "ray", img)[0, 0]
    u = (np.arange(64) - 31.5) * 0.5
    # block faces: y in [-8, 4), x in [-6, 6); ray x(y) = u (500 - y) / 1000
    xa = u * (500 - 4) / 1000
    xb = u * (500 + 8) / 1000
    inside = (np.abs(xa) < 6) & (np.abs(xb) < 6)
    np.testing.assert_allclose(y[inside], (mu * 12 * np.sqrt(1 + (u / 1000) ** 2))[inside], rtol=1e-13)


def test_disk_converges_to_analytic_chord():
    """Uniform disk (radius 20 mm, mu = 0.02): the ray-driven projection of
    the voxelised disk tends to 2 mu sqrt(r^2 - d^2) as the pixel shrinks."""
    r, mu, fov = 20.0, 0.02, 64.0
    errs = []
    for n in (32, 64, 128, 256):
        h = fov / n
        spec = W.GeometrySpec("fan2d", "flat", n, n, 1, h, h, 1.0, 101, 1, 0.7, 1.0, 1,
                              theta=0.37, sad=400.0, sdd=800.0)
        c = (np.arange(n) - (n - 1) / 2) * h
        X, Y = np.meshgrid(c, c)
        img = np.where(X ** 2 + Y ** 2 <= r * r, mu, 0.0)[None]
        y = oracle.forward(spec, "ray", img)[0, 0]
        f = oracle.frame(spec, 0)
        want = np.zeros(101)
        for a in range(101):
            P = oracle.cell_point(spec, 0, a, 0)
            d = P - f["s"]
            dist = np.linalg.norm(np.cross(d, -f["s"])) / np.linalg.norm(d)
            want[a] = 2 * mu * math.sqrt(max(r * r - dist * dist, 0.0))
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.01


def _quadric_chord(s, d, c, Q):
    """Length of the line s + t d inside the quadric (X - c)^T Q (X - c) <= 1:
    with alpha = d^T Q d, beta = d^T Q (s - c), gamma = (s - c)^T Q (s - c),
    the roots of alpha t^2 + 2 beta t + gamma - 1 = 0 are 2 sqrt(beta^2 -
    alpha (gamma - 1)) / alpha apart in t, i.e. that times |d| in mm."""
    w = s - c
    alpha, beta, gamma = d @ Q @ d, d @ Q @ w, w @ Q @ w
    disc = beta * beta - alpha * (gamma - 1.0)
    return 2.0 * math.sqrt(disc) / alpha * np.linalg.norm(d) if disc > 0 else 0.0


def _rotation(a, b, c):
    """Rotation matrix from z-y-x angles (radians)."""
    ca, sa, cb, sb, cc, sc = math.cos(a), math.sin(a), math.cos(b), math.sin(b), math.cos(c), math.sin(c)
    Rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1]])
    Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
    Rx = np.array([[1, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return Rz @ Ry @ Rx


def _converges(errs, final, rate=None):
    """Errors fall with every refinement, below `final` at the finest grid;
    with `rate`, each halving of the voxel divides the error by at least
    that factor (a voxelised boundary converges at first order in h)."""
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    if rate is not None:
        assert all(e0 / e1 > rate for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < final, errs


def test_ellipse_converges_to_analytic_chord():
    """Uniform ellipse (semi-axes 22 and 12 mm, rotated 0.6 rad, centred at
    (6, -4) mm, mu = 0.02): the ray-driven projection of the voxelised
    ellipse tends to mu times the line's chord through the ellipse."""
    mu, fov = 0.02, 64.0
    c = np.array([6.0, -4.0, 0.0])
    R = _rotation(0.6, 0.0, 0.0)
    Q = R @ np.diag([1 / 22.0 ** 2, 1 / 12.0 ** 2, 0.0]) @ R.T
    errs = []
    for n in (32, 64, 128, 256):
        h = fov / n
        spec = W.GeometrySpec("fan2d", "flat", n, n, 1, h, h, 1.0, 101, 1, 0.7, 1.0, 1,
                              theta=1.1, sad=400.0, sdd=800.0)
        g = (np.arange(n) - (n - 1) / 2) * h
        X, Y = np.meshgrid(g, g)
        P = np.stack([X - c[0], Y - c[1], np.zeros_like(X)], axis=-1)
        img = np.where(np.einsum("...i,ij,...j->...", P, Q, P) <= 1.0, mu, 0.0)[None]
        y = oracle.forward(spec, "ray", img)[0, 0]
        s = oracle.frame(spec, 0)["s"]
        want = np.array([mu * _quadric_chord(s, oracle.cell_point(spec, 0, a, 0) - s, c, Q) for a in range(101)])
        assert (want > 0).sum() > 30
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    _converges(errs, 0.01, rate=1.6)


def _solid_3d(kind, quadric, c, mu, n, fov, nu, nv, du, **kw):
    h = fov / n
    spec = W.GeometrySpec(kind, "flat", n, n, n, h, h, h, nu, nv, du, du, 1, sad=300.0, sdd=600.0, **kw)
    g = (np.arange(n) - (n - 1) / 2) * h
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X - c[0], Y - c[1], Z - c[2]], axis=-1)
    img = np.where(np.einsum("...i,ij,...j->...", P, quadric, P) <= 1.0, mu, 0.0)
    y = oracle.forward(spec, "ray", img)[0]
    s = oracle.frame(spec, 0)["s"]
    want = np.array([[mu * _quadric_chord(s, oracle.cell_point(spec, 0, a, b) - s, c, quadric)
                      for a in range(nu)] for b in range(nv)])
    return y, want


def test_ball_converges_to_analytic_chord_3d():
    """Uniform ball (radius 18 mm at (5, -3, 4) mm, mu = 0.02) in circular cone
    beam: the projection of the voxelised ball tends to 2 mu sqrt(r^2 - d^2),
    d the distance from the ball's centre to the ray."""
    r, mu = 18.0, 0.02
    c = np.array([5.0, -3.0, 4.0])
    errs = []
    for n in (16, 32, 64, 128):
        y, want = _solid_3d("circ3d", np.eye(3) / r ** 2, c, mu, n, 64.0, 27, 21, 3.0, theta=0.5)
        assert (want > 0).sum() > 150
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    _converges(errs, 0.025, rate=1.6)


def test_ellipsoid_converges_to_analytic_chord_noncircular():
    """Uniform ellipsoid (semi-axes 20, 14, 10 mm, rotated, off centre) seen
    from a tilted, rolled non-circular pose: the projection of the voxelised
    ellipsoid tends to mu times the line's chord through the ellipsoid."""
    mu = 0.02
    c = np.array([-4.0, 3.0, -2.0])
    R = _rotation(0.4, -0.7, 0.3)
    Q = R @ np.diag([1 / 20.0 ** 2, 1 / 14.0 ** 2, 1 / 10.0 ** 2]) @ R.T
    errs = []
    for n in (16, 32, 64, 128):
        y, want = _solid_3d("noncirc3d", Q, c, mu, n, 64.0, 27, 21, 3.0, theta=2.2, phi=0.15, psi=0.1,
                            z_src=3.0, u_ofst=1.5, v_ofst=-2.0)
        assert (want > 0).sum() > 100
        errs.append(np.linalg.norm(y - want) / np.linalg.norm(want))
    _converges(errs, 0.025, rate=1.6)
