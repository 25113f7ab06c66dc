"""Pins of the oracle's "recon" mode (filtered backprojection, Sec. 2.3):
the discrete ramp's frequency response, the angular weights, and FBP of
objects whose projections are known in closed form (chords through a disk
or a ball), reconstructed back to their value."""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _analytic_sino(spec, centre, radius, mu):
    """Line integrals of a uniform ball (disk in 2D) along the ray from the
    source to every cell centre: mu * 2 sqrt(r^2 - d^2)."""
    nv = 1 if spec.kind == "fan2d" else spec.nv
    ua = (np.arange(spec.nu) - 0.5 * (spec.nu - 1)) * spec.du
    vb = (np.arange(nv) - 0.5 * (nv - 1)) * (1.0 if spec.kind == "fan2d" else spec.dv)
    out = np.zeros((spec.nview, nv, spec.nu))
    c0 = np.asarray(centre, dtype=np.float64)
    for v in range(spec.nview):
        f = oracle.frame(spec, v)
        U, V = np.meshgrid(ua, vb)
        if spec.det == "curved":
            gam = (f["u0"] + U) / f["D"]
            P = (f["s"][None, None, :] + f["D"] * (np.cos(gam)[..., None] * f["n"] + np.sin(gam)[..., None] * f["eu"])
                 + (f["h0"] + V)[..., None] * f["ev"])
        else:
            P = f["c"][None, None, :] + U[..., None] * f["eu"] + V[..., None] * f["ev"]
        d = P - f["s"]
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        w = c0 - f["s"]
        t = w @ np.eye(3)
        proj = (d * t).sum(-1)
        dist2 = (w * w).sum() - proj ** 2
        out[v] = mu * 2.0 * np.sqrt(np.maximum(radius ** 2 - dist2, 0.0))
    return out


def test_ramp_response_is_half_the_ramp():
    """Impulse response of the flat-detector filter at the principal point:
    its Fourier transform is |f| / 2 up to the Nyquist frequency (the FBP
    over the full circle counts every line twice)."""
    nu, du = 1025, 0.8
    spec = W.GeometrySpec("fan2d", "flat", 4, 4, 1, 1.0, 1.0, 1.0, nu, 1, du, 1.0, 1, theta=0.0,
                          sad=500.0, sdd=1000.0)
    # a unit sample at the principal point: q[m] = du h(u_m), and the filter's
    # transfer function is H(f) = du sum_m h(u_m) cos(2 pi f u_m) = sum_m q[m] cos(..)
    y = np.zeros((1, 1, nu))
    y[0, 0, nu // 2] = 1.0
    q = oracle.ramp_filter(spec, y)[0, 0]
    k = (np.arange(nu) - nu // 2) * du
    for f in (0.0, 0.05, 0.2, 0.4, 0.6):
        H = float(np.sum(q * np.cos(2 * np.pi * f * k)))
        assert abs(H - abs(f) / 2) < 2e-3, (f, H)


def test_angular_weights_cover_the_circle():
    rng = np.random.default_rng(3)
    th = np.sort(rng.uniform(0, 2 * np.pi, 37))
    spec = W.GeometrySpec("fan2d", "flat", 4, 4, 1, 1.0, 1.0, 1.0, 8, 1, 1.0, 1.0, 37, theta=th,
                          sad=500.0, sdd=1000.0)
    w = np.array([oracle.recon_dbeta(spec, v) for v in range(37)])
    assert abs(w.sum() - 2 * np.pi) < 1e-12
    eq = W.GeometrySpec("fan2d", "flat", 4, 4, 1, 1.0, 1.0, 1.0, 8, 1, 1.0, 1.0, 90,
                        theta=np.linspace(0, 2 * np.pi, 90, endpoint=False), sad=500.0, sdd=1000.0)
    assert all(abs(oracle.recon_dbeta(eq, v) - 2 * np.pi / 90) < 1e-12 for v in range(90))


@pytest.mark.parametrize("det", ["flat", "curved"])
@pytest.mark.parametrize("centre", [(0.0, 0.0), (12.0, -7.0)])
def test_fan_fbp_reconstructs_a_uniform_disk(det, centre):
    n, nview, mu, r = 128, 360, 0.02, 30.0
    spec = W.GeometrySpec("fan2d", det, n, n, 1, 1.0, 1.0, 1.0, 384, 1, 0.8, 1.0, nview,
                          theta=np.linspace(0, 2 * np.pi, nview, endpoint=False), sad=500.0, sdd=1000.0)
    y = _analytic_sino(spec, (centre[0], centre[1], 0.0), r, mu)
    x = oracle.fbp(spec, y)[0]
    c = np.arange(n) - 0.5 * (n - 1)
    yy, xx = np.meshgrid(c, c, indexing="ij")
    d = np.hypot(xx - centre[0], yy - centre[1])
    inside, outside = x[d < 0.7 * r], x[(d > 1.3 * r) & (np.hypot(xx, yy) < 55)]
    assert abs(inside.mean() - mu) < 0.01 * mu, inside.mean()
    assert np.abs(inside - mu).max() < 0.05 * mu
    assert abs(outside.mean()) < 0.02 * mu and np.abs(outside).max() < 0.1 * mu


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_fdk_reconstructs_the_central_slice_of_a_ball(det):
    n, nview, mu, r = 64, 180, 0.02, 20.0
    spec = W.GeometrySpec("circ3d", det, n, n, n, 1.0, 1.0, 1.0, 160, 120, 1.0, 1.0, nview,
                          theta=np.linspace(0, 2 * np.pi, nview, endpoint=False), sad=400.0, sdd=800.0)
    y = _analytic_sino(spec, (0.0, 0.0, 0.0), r, mu)
    x = oracle.fbp(spec, y)
    c = np.arange(n) - 0.5 * (n - 1)
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    d = np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    mid = np.abs(zz) < 1.0  # the two slices next to the mid-plane
    inside = x[mid & (d < 0.7 * r)]
    assert abs(inside.mean() - mu) < 0.015 * mu, inside.mean()
    assert np.abs(x[mid & (d > 1.3 * r) & (np.hypot(xx, yy) < 28)]).mean() < 0.02 * mu


def _gauss_cyl_sino(spec, centre, sigma, mu):
    """Line integrals of the z-invariant Gaussian mu exp(-|xy - c|^2 / 2 s^2)
    (a 2D Gaussian in the fan plane): along a ray of unit direction d,
    mu sqrt(2 pi) sigma exp(-dist^2 / 2 s^2) / |d_xy|, dist = distance from
    the axis to the ray's projection on the xy plane."""
    nv = 1 if spec.kind == "fan2d" else spec.nv
    ua = (np.arange(spec.nu) - 0.5 * (spec.nu - 1)) * spec.du
    vb = (np.arange(nv) - 0.5 * (nv - 1)) * (1.0 if spec.kind == "fan2d" else spec.dv)
    out = np.zeros((spec.nview, nv, spec.nu))
    c0 = np.asarray(centre, dtype=np.float64)
    for v in range(spec.nview):
        f = oracle.frame(spec, v)
        U, V = np.meshgrid(ua, vb)
        if spec.det == "curved":
            gam = (f["u0"] + U) / f["D"]
            P = (f["s"] + f["D"] * (np.cos(gam)[..., None] * f["n"] + np.sin(gam)[..., None] * f["eu"])
                 + (f["h0"] + V)[..., None] * f["ev"])
        else:
            P = f["c"] + U[..., None] * f["eu"] + V[..., None] * f["ev"]
        d = P - f["s"]
        d /= np.linalg.norm(d, axis=-1, keepdims=True)
        dxy = np.hypot(d[..., 0], d[..., 1])
        e = d[..., :2] / dxy[..., None]  # unit direction of the projected line
        w = c0[:2] - f["s"][:2]
        along = e[..., 0] * w[0] + e[..., 1] * w[1]
        dist2 = w @ w - along ** 2
        out[v] = mu * math.sqrt(2 * math.pi) * sigma * np.exp(-dist2 / (2 * sigma ** 2)) / dxy
    return out


def _uneven_angles(n):
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    return t + 0.5 * np.sin(t)  # views denser on one side of the circle


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_fan_fbp_reconstructs_an_off_centre_gaussian(det):
    """Wide fan (object shadow up to ~14 deg off the principal ray), a
    detector offset of 90 mm (the weights are taken about the principal
    point, not the detector centre), uneven view angles, no truncation: FBP
    of a smooth object matches it to 0.5 % of its peak."""
    n, nview, mu, sigma, c = 128, 240, 0.02, 6.0, (38.0, -24.0)
    spec = W.GeometrySpec("fan2d", det, n, n, 1, 1.0, 1.0, 1.0, 1000, 1, 0.5, 1.0, nview,
                          theta=_uneven_angles(nview), sad=250.0, sdd=500.0, u_ofst=90.0)
    y = _gauss_cyl_sino(spec, (c[0], c[1], 0.0), sigma, mu)
    x = oracle.fbp(spec, y)[0]
    g = np.arange(n) - 0.5 * (n - 1)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    ref = mu * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / (2 * sigma ** 2))
    roi = np.hypot(xx, yy) < 60
    assert np.abs(x - ref)[roi].max() < 0.005 * mu, np.abs(x - ref)[roi].max() / mu


@pytest.mark.parametrize("det", ["flat", "curved"])
def test_fdk_is_exact_for_a_z_invariant_object(det):
    """FDK reconstructs an object that does not vary along z at every slice
    (the tilted-fan weights make each row a consistent fan): a Gaussian
    cylinder over 48 slices, cone half-angle ~12 deg, detector offsets in u
    and v."""
    nx, nz, nview, mu, sigma, c = 48, 48, 180, 0.02, 5.0, (8.0, -5.0)
    spec = W.GeometrySpec("circ3d", det, nx, nx, nz, 1.0, 1.0, 1.0, 160, 176, 0.8, 1.0, nview,
                          theta=_uneven_angles(nview), sad=200.0, sdd=400.0, u_ofst=8.0, v_ofst=15.0)
    y = _gauss_cyl_sino(spec, (c[0], c[1], 0.0), sigma, mu)
    x = oracle.fbp(spec, y)
    g = np.arange(nx) - 0.5 * (nx - 1)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    ref = mu * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / (2 * sigma ** 2))
    roi = np.hypot(xx, yy) < 20
    err = max(np.abs(x[k] - ref)[roi].max() for k in range(nz))
    assert err < 0.005 * mu, err / mu


@pytest.mark.parametrize("proj", ["dd", "sf"])
@pytest.mark.parametrize("det", ["flat", "curved"])
def test_footprint_recon_backprojections_reconstruct_the_gaussian(proj, det):
    """Recon mode with the normalised DD / SF footprints as the interpolation:
    the z-invariant Gaussian cylinder comes back at every slice (to 1 % of
    its peak: the footprints smooth a little more than the bilinear hat)."""
    nx, nz, nview, mu, sigma, c = 48, 24, 180, 0.02, 5.0, (8.0, -5.0)
    spec = W.GeometrySpec("circ3d", det, nx, nx, nz, 1.0, 1.0, 1.0, 160, 96, 0.8, 1.0, nview,
                          theta=_uneven_angles(nview), sad=200.0, sdd=400.0, u_ofst=8.0, v_ofst=15.0)
    y = _gauss_cyl_sino(spec, (c[0], c[1], 0.0), sigma, mu)
    x = oracle.fbp(spec, y, proj)
    g = np.arange(nx) - 0.5 * (nx - 1)
    yy, xx = np.meshgrid(g, g, indexing="ij")
    ref = mu * np.exp(-((xx - c[0]) ** 2 + (yy - c[1]) ** 2) / (2 * sigma ** 2))
    roi = np.hypot(xx, yy) < 20
    err = max(np.abs(x[k] - ref)[roi].max() for k in range(nz))
    assert err < 0.01 * mu, err / mu


@pytest.mark.parametrize("proj", ["dd", "sf"])
def test_footprint_recon_weights_interpolate_constants(proj):
    """The normalised footprint weights of a voxel whose footprint lies on
    the detector sum to 1: a constant filtered sinogram backprojects to the
    sum of the depth weights, the same as with the bilinear hat."""
    spec = W.GeometrySpec("circ3d", "flat", 6, 6, 6, 1.0, 1.0, 1.0, 40, 40, 1.0, 1.0, 5,
                          theta=np.linspace(0, 2 * np.pi, 5, endpoint=False), sad=60.0, sdd=120.0)
    q = np.ones(spec.sino_shape)
    np.testing.assert_allclose(oracle.back_recon(spec, q, proj), oracle.back_recon(spec, q, "voxel"),
                               rtol=1e-12)
