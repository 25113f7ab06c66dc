"""Pins of the oracle's voxel-driven, distance-driven and separable-footprint
projectors (Sec. 2.3: Peters 1981, De Man & Basu 2004, Long et al. 2010).

Closed forms used here are derived by hand in the docstrings.  'Parallel
limit' geometries put source and detector very far away (Sec. 2.2: a parallel
beam is a divergent beam with very large SAD and SDD).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from brute import subray_average_parallel_2d

# Parallel limit.  At theta = 0 the source offset cancels exactly, so a very
# far source is exact to rounding; at oblique angles w = X - s cancels about
# FAR * 1e-16, and FAR = 1e9 balances that against the residual perspective
# (~1e-7 relative), so those checks use rel = 1e-6.
FAR = 1.0e12
FAR_OBLIQUE = 1.0e9
REL_OBLIQUE = 1e-6


def parallel_2d(n=16, h=1.0, nu=None, du=None, theta=0.0, nview=1):
    nu = nu or n
    du = du or h
    far = FAR if theta == 0.0 else FAR_OBLIQUE
    return W.GeometrySpec("fan2d", "flat", n, n, 1, h, h, 1.0, nu, 1, du, 1.0, nview,
                          theta=theta, sad=far, sdd=far + 100.0)


# ------------------------------------------------------------------ voxel-driven

def test_voxel_single_voxel_closed_form_2d():
    """Voxel at the origin, theta = 0, nu even: the centre projects midway
    between cells nu/2-1 and nu/2, each gets half the amplitude
    dx dy r SDD / (depth^2 du) with r = depth = SAD."""
    spec = W.GeometrySpec("fan2d", "flat", 5, 5, 1, 2.0, 3.0, 1.0, 8, 1, 1.7, 1.0, 1,
                          theta=0.0, sad=400.0, sdd=900.0)
    a, b, w = oracle.footprint(spec, "voxel", 0, 2, 2, 0)
    amp = 2.0 * 3.0 * 900.0 / (400.0 * 1.7)
    assert sorted(a.tolist()) == [3, 4]
    np.testing.assert_allclose(w, [amp / 2, amp / 2], rtol=1e-14)


def test_voxel_single_voxel_closed_form_3d():
    """3D: amplitude V r SDD^2 / (depth^3 du dv) = V SDD^2 / (SAD^2 du dv),
    split equally over the four cells around the centre (nu, nv even)."""
    spec = W.GeometrySpec("circ3d", "flat", 3, 3, 3, 1.0, 2.0, 0.5, 6, 4, 1.5, 1.2, 1,
                          theta=0.0, sad=500.0, sdd=1000.0)
    a, b, w = oracle.footprint(spec, "voxel", 0, 1, 1, 1)
    amp = 1.0 * 2.0 * 0.5 * 1000.0 ** 2 / (500.0 ** 2 * 1.5 * 1.2)
    assert sorted(zip(a.tolist(), b.tolist())) == [(2, 1), (2, 2), (3, 1), (3, 2)]
    np.testing.assert_allclose(w, [amp / 4] * 4, rtol=1e-14)


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_voxel_off_axis_closed_form_3d(det):
    """Off-axis voxel at (40, 0, 30) under theta = 0, SAD 500, SDD 1000, so
    w = (40, -500, 30), r = sqrt(252500).  Flat: depth = w.n = 500, amplitude
    V r SDD^2 / (depth^3 du dv).  Curved: rho = sqrt(40^2 + 500^2), amplitude
    V r SDD^2 / (rho^3 du dv).  (Point mass over the ray density there.)"""
    spec = W.GeometrySpec("circ3d", det, 3, 1, 3, 40.0, 10.0, 30.0, 128, 96, 2.0, 2.0, 1,
                          theta=0.0, sad=500.0, sdd=1000.0)
    _, _, w = oracle.footprint(spec, "voxel", 0, 2, 0, 2)
    r = math.sqrt(252500.0)
    rho = 500.0 if det == "flat" else math.sqrt(40.0 ** 2 + 500.0 ** 2)
    want = 40.0 * 10.0 * 30.0 * r * 1e6 / (rho ** 3 * 4.0)
    assert w.sum() == pytest.approx(want, rel=1e-13)


def test_voxel_off_axis_closed_form_2d():
    """2D: pixel at (40, 0): r = sqrt(40^2 + 500^2), depth 500, amplitude
    dx dy r SDD / (depth^2 du)."""
    spec = W.GeometrySpec("fan2d", "flat", 3, 1, 1, 40.0, 10.0, 1.0, 128, 1, 2.0, 1.0, 1,
                          theta=0.0, sad=500.0, sdd=1000.0)
    _, _, w = oracle.footprint(spec, "voxel", 0, 2, 0, 0)
    want = 40.0 * 10.0 * math.sqrt(40.0 ** 2 + 500.0 ** 2) * 1000.0 / (500.0 ** 2 * 2.0)
    assert w.sum() == pytest.approx(want, rel=1e-13)


def test_voxel_curved_amplitude_closed_form():
    """Curved 2D: amplitude dx dy SDD / (rho du) where rho is the voxel's
    distance from the source; a voxel at (0, 0) under theta = 0 has rho = SAD."""
    spec = W.GeometrySpec("fan2d", "curved", 5, 5, 1, 2.0, 2.0, 1.0, 8, 1, 1.1, 1.0, 1,
                          theta=0.0, sad=450.0, sdd=1000.0)
    _, _, w = oracle.footprint(spec, "voxel", 0, 2, 2, 0)
    assert w.sum() == pytest.approx(4.0 * 1000.0 / (450.0 * 1.1), rel=1e-14)


def test_voxel_bilinear_partition_of_unity():
    """The bilinear weights of a voxel sum to one, so the footprint weights
    split the amplitude in the ratio given by the projected position."""
    spec = W.scaled(W.circ3d_256(), 16, 5)
    for v in range(5):
        for (i, j, k) in [(3, 7, 2), (10, 12, 9), (8, 8, 8)]:
            a, b, w = oracle.footprint(spec, "voxel", v, i, j, k)
            assert len(w) == 4
            X = [(i - 7.5) * spec.dx, (j - 7.5) * spec.dy, (k - (spec.nz - 1) / 2) * spec.dz]
            u, vv = oracle.project(spec, v, X)
            fu = u / spec.du + (spec.nu - 1) / 2
            fv = vv / spec.dv + (spec.nv - 1) / 2
            tot = w.sum()
            wa = w[a == a.max()].sum() / tot
            wb = w[b == b.max()].sum() / tot
            assert wa == pytest.approx(fu - math.floor(fu), abs=1e-12)
            assert wb == pytest.approx(fv - math.floor(fv), abs=1e-12)


def test_voxel_parallel_limit_mass():
    """Parallel limit: the weights of any pixel sum to dx dy / du."""
    spec = parallel_2d(n=12, h=1.5, nu=40, du=0.9, theta=0.63)
    for (i, j) in [(0, 0), (5, 7), (11, 3)]:
        _, _, w = oracle.footprint(spec, "voxel", 0, i, j, 0)
        assert w.sum() == pytest.approx(1.5 * 1.5 / 0.9, rel=REL_OBLIQUE)


# ------------------------------------------------------------------ distance-driven

def test_dd_parallel_aligned_equals_column_sums():
    """theta = 0 parallel limit, du = dx, detector aligned with the pixel
    columns: each cell collects exactly its column, y = dy sum_j x[j, a]."""
    spec = parallel_2d(n=16, h=1.25)
    x = W.random_volume(spec, 2)[0]
    y = oracle.forward(spec, "dd", x)[0, 0]
    np.testing.assert_allclose(y, 1.25 * x[0].sum(axis=0), rtol=1e-9)


def test_dd_parallel_aligned_at_90_deg_equals_row_sums():
    """theta = 90 deg: the main axis is x; e_u = (0, 1), so cell a collects
    row a: y = dx sum_i x[a, i]."""
    spec = parallel_2d(n=16, h=0.75, theta=math.pi / 2)
    x = W.random_volume(spec, 3)[0]
    y = oracle.forward(spec, "dd", x)[0, 0]
    np.testing.assert_allclose(y, 0.75 * x[0].sum(axis=1), rtol=REL_OBLIQUE)


def test_dd_parallel_aligned_3d_equals_column_sums():
    spec = W.GeometrySpec("circ3d", "flat", 8, 9, 6, 1.0, 0.5, 2.0, 8, 6, 1.0, 2.0, 1,
                          theta=0.0, sad=FAR, sdd=FAR + 100.0)
    x = W.random_volume(spec, 5)[0]
    y = oracle.forward(spec, "dd", x)[0]
    np.testing.assert_allclose(y, 0.5 * x.sum(axis=1), rtol=1e-9)


@pytest.mark.parametrize("theta", [0.0, 0.3, -0.6, math.pi - 0.2])
def test_dd_parallel_mass(theta):
    """Parallel limit, main axis y: overlaps sum to dx |cos t| and the slab
    path is dy / |cos t|, so the weights of a pixel sum to dx dy / du."""
    spec = parallel_2d(n=10, h=1.0, nu=64, du=0.37, theta=theta)
    for (i, j) in [(0, 0), (4, 6), (9, 2)]:
        _, _, w = oracle.footprint(spec, "dd", 0, i, j, 0)
        assert w.sum() == pytest.approx(1.0 / 0.37, rel=REL_OBLIQUE)


def test_dd_fan_partition_of_boundaries():
    """Fan beam: sum_c overlap_c = u+ - u- where u+- are the projections of
    the pixel's boundary points on the slab line (main axis y at theta=0.2);
    with L_c divided out, the weights recover that width."""
    spec = W.GeometrySpec("fan2d", "flat", 9, 9, 1, 2.0, 2.0, 1.0, 64, 1, 0.8, 1.0, 1,
                          theta=0.2, sad=300.0, sdd=700.0)
    f = oracle.frame(spec, 0)
    for (i, j) in [(1, 1), (4, 4), (7, 2)]:
        a, b, w = oracle.footprint(spec, "dd", 0, i, j, 0)
        X = np.array([(i - 4) * 2.0, (j - 4) * 2.0, 0.0])
        u1 = oracle.project(spec, 0, X - [1.0, 0, 0])[0]
        u2 = oracle.project(spec, 0, X + [1.0, 0, 0])[0]
        Lc = []
        for aa in a:
            P = oracle.cell_point(spec, 0, int(aa), 0)
            d = P - f["s"]
            Lc.append(2.0 * np.linalg.norm(d) / abs(d[1]))
        assert (w / np.array(Lc)).sum() * 0.8 == pytest.approx(abs(u2 - u1), rel=1e-12)


# ------------------------------------------------------------------ separable footprint

@pytest.mark.parametrize("theta", [0.0, 0.25, math.pi / 4, 1.1, 2.5])
def test_sf_parallel_mass_2d(theta):
    """Parallel limit: trapezoid area (|c|+|s| + ||c|-|s||) dx / 2 =
    dx max(|c|, |s|) times amplitude dx / max(|c|, |s|) gives sum w du = dx dy."""
    spec = parallel_2d(n=10, h=1.3, nu=60, du=0.41, theta=theta)
    for (i, j) in [(0, 0), (3, 8), (9, 5)]:
        _, _, w = oracle.footprint(spec, "sf", 0, i, j, 0)
        assert w.sum() * 0.41 == pytest.approx(1.3 * 1.3, rel=REL_OBLIQUE)


def test_sf_parallel_mass_3d():
    spec = W.GeometrySpec("circ3d", "flat", 6, 6, 6, 1.0, 1.0, 0.7, 40, 30, 0.45, 0.33, 1,
                          theta=0.7, sad=FAR_OBLIQUE, sdd=FAR_OBLIQUE + 100.0)
    for (i, j, k) in [(0, 0, 0), (2, 3, 4), (5, 1, 5)]:
        _, _, w = oracle.footprint(spec, "sf", 0, i, j, k)
        assert w.sum() * 0.45 * 0.33 == pytest.approx(1.0 * 1.0 * 0.7, rel=REL_OBLIQUE)


@pytest.mark.parametrize("theta", [0.3, math.pi / 4, 2.0])
def test_sf_parallel_is_exact_pixel_projection(theta):
    """In the parallel limit the SF trapezoid is the exact projection of a
    square pixel, so SF equals the cell average of exact line integrals,
    here from 4000 brute-force sub-rays per cell."""
    spec = parallel_2d(n=6, h=2.0, nu=24, du=0.9, theta=theta)
    x = W.random_volume(spec, 7)[0]
    y = oracle.forward(spec, "sf", x)[0, 0]
    ref = subray_average_parallel_2d(spec, x[0], 0, 4000)
    np.testing.assert_allclose(y, ref, rtol=0, atol=2e-6 * np.abs(ref).max())


def test_sf_equals_dd_at_zero_angle_parallel():
    spec = parallel_2d(n=12, h=1.0, nu=30, du=0.55)
    x = W.random_volume(spec, 8)[0]
    np.testing.assert_allclose(oracle.forward(spec, "sf", x), oracle.forward(spec, "dd", x),
                               rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_sf_fan_trapezoid_area(det):
    """Fan beam: for a voxel inside the detector, sum_c w du = l * area where
    area = (t3 + t2 - t1 - t0) / 2 from the projected column corners and
    l = dx |w| / max(|w_x|, |w_y|)."""
    spec = W.GeometrySpec("fan2d", det, 9, 9, 1, 2.0, 2.0, 1.0, 80, 1, 0.7, 1.0, 1,
                          theta=0.9, sad=300.0, sdd=700.0, x_src=2.0, u_ofst=1.0)
    f = oracle.frame(spec, 0)
    for (i, j) in [(0, 8), (4, 4), (7, 1)]:
        X = np.array([(i - 4) * 2.0, (j - 4) * 2.0, 0.0])
        t = sorted(oracle.project(spec, 0, X + [sx, sy, 0.0])[0]
                   for sx in (-1.0, 1.0) for sy in (-1.0, 1.0))
        area = (t[3] + t[2] - t[1] - t[0]) / 2
        w_ = X - f["s"]
        amp = 2.0 * np.linalg.norm(w_) / max(abs(w_[0]), abs(w_[1]))
        _, _, w = oracle.footprint(spec, "sf", 0, i, j, 0)
        assert w.sum() * 0.7 == pytest.approx(amp * area, rel=1e-12)


def test_sf_degenerate_trapezoid_is_finite():
    """At 45 deg in the parallel limit two corners coincide in pairs
    (triangle); at 0 deg too (rectangle).  No division by a zero width."""
    for theta in (0.0, math.pi / 4, math.pi / 2):
        spec = parallel_2d(n=4, h=1.0, nu=16, du=0.5, theta=theta)
        _, _, w = oracle.footprint(spec, "sf", 0, 1, 2, 0)
        assert np.all(np.isfinite(w)) and w.sum() * 0.5 == pytest.approx(1.0, rel=REL_OBLIQUE)
