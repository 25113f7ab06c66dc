"""Pins of the oracle's ray-driven projector (Siddon 1985, Sec. 2.3).

* all-pairs brute force (slab method per ray and voxel, no traversal);
* closed-form chords through the volume box and through grid-aligned blocks;
* convergence of a voxelised disk to the analytic chord 2 mu sqrt(r^2 - d^2).
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
