"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds data only: scan-geometry parameter sets (what a user passes
to the geometry constructor), seeded random phantoms and sinograms, and the
named workload shapes.  It contains none of the projection arithmetic (no
rotation, no detector mapping, no footprint): the oracle and the CUDA library
each implement that on their own from the parameters defined here.

Geometry parameters follow the paper's parameter table (Sec. 2.2, Table 1):
gantry angle theta, off-plane phi, in-plane psi, SAD, SDD, source offsets
(x_src, z_src), object offsets (x_ofst, y_ofst, z_ofst) and detector offsets
(u_ofst, v_ofst).  Every parameter is a scalar shared by all views or a vector
of one value per view (Sec. 2.2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

KINDS = ("fan2d", "circ3d", "noncirc3d")
DETS = ("flat", "curved")
PER_VIEW = ("theta", "phi", "psi", "sad", "sdd", "x_src", "z_src",
            "x_ofst", "y_ofst", "z_ofst", "u_ofst", "v_ofst")


@dataclasses.dataclass
class GeometrySpec:
    """Scanner geometry parameters (Sec. 2.2, Table 1).  Angles in radians,
    lengths in mm.  For 'fan2d', nz = nv = 1 and dz, dv, z_*, v_ofst, phi and
    psi are unused.  `poses` (nview x 12: source xyz, detector-centre xyz, e_u
    xyz, e_v xyz) replaces the angle parametrisation for 'noncirc3d'."""
    kind: str
    det: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    nu: int
    nv: int
    du: float
    dv: float
    nview: int
    theta: object = 0.0
    phi: object = 0.0
    psi: object = 0.0
    sad: object = 500.0
    sdd: object = 1000.0
    x_src: object = 0.0
    z_src: object = 0.0
    x_ofst: object = 0.0
    y_ofst: object = 0.0
    z_ofst: object = 0.0
    u_ofst: object = 0.0
    v_ofst: object = 0.0
    poses: Optional[np.ndarray] = None

    def __post_init__(self):
        if self.kind not in KINDS:
            raise ValueError(f"kind must be one of {KINDS}")
        if self.det not in DETS:
            raise ValueError(f"det must be one of {DETS}")

    # -- data access -------------------------------------------------------
    def param(self, name: str) -> np.ndarray:
        """The raw parameter as a float64 array of length 1 or nview."""
        a = np.atleast_1d(np.asarray(getattr(self, name), dtype=np.float64))
        return np.ascontiguousarray(a.ravel())

    def per_view(self, name: str) -> np.ndarray:
        """The parameter repeated to one value per view."""
        a = self.param(name)
        if a.size == 1:
            return np.full(self.nview, a[0])
        if a.size != self.nview:
            raise ValueError(f"{name}: length {a.size} is neither 1 nor nview={self.nview}")
        return a.copy()

    def subset(self, views: Sequence[int]) -> "GeometrySpec":
        """The same scan restricted to the listed views (an ordered subset)."""
        views = np.asarray(views, dtype=np.int64)
        kw = dataclasses.asdict(self)
        kw["nview"] = int(views.size)
        for name in PER_VIEW:
            a = self.param(name)
            kw[name] = a.copy() if a.size == 1 else a[views].copy()
        if self.poses is not None:
            kw["poses"] = np.ascontiguousarray(np.asarray(self.poses)[views])
        return GeometrySpec(**kw)

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def sino_shape(self):
        return (self.nview, self.nv, self.nu)

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_cells(self) -> int:
        return self.nview * self.nv * self.nu


def _angles(nview: int, span: float = 2 * math.pi, start: float = 0.0) -> np.ndarray:
    return start + span * np.arange(nview, dtype=np.float64) / nview


# -- named workloads -----------------------------------------------------------

def fan2d_small(nview: int = 180) -> GeometrySpec:
    """2D fan beam: 128x128 image of 1 mm pixels, 180 views over 360 deg,
    flat 256-bin detector of 1.2 mm, SAD 500 mm, SDD 1000 mm."""
    return GeometrySpec("fan2d", "flat", 128, 128, 1, 1.0, 1.0, 1.0,
                        256, 1, 1.2, 1.0, nview, theta=_angles(nview),
                        sad=500.0, sdd=1000.0)


def circ3d_256(nview: int = 360) -> GeometrySpec:
    """3D circular cone beam: 256^3 volume of 0.5 mm voxels, 360 views over
    360 deg, flat 512x384 detector of 0.8 mm, SAD 785 mm, SDD 1085 mm."""
    return GeometrySpec("circ3d", "flat", 256, 256, 256, 0.5, 0.5, 0.5,
                        512, 384, 0.8, 0.8, nview, theta=_angles(nview),
                        sad=785.0, sdd=1085.0)


def circ3d_curved(nview: int = 984) -> GeometrySpec:
    """3D circular cone beam with a curved (cylindrical) 888x64 detector of
    1.0 mm arc cells, 984 views, 512x512x128 volume of 0.8x0.8x0.25 mm,
    SAD 595 mm, SDD 1085.6 mm."""
    return GeometrySpec("circ3d", "curved", 512, 512, 128, 0.8, 0.8, 0.25,
                        888, 64, 1.0, 1.0, nview, theta=_angles(nview),
                        sad=595.0, sdd=1085.6)


def noncirc3d_saddle(nview: int = 500, n: int = 512, ndet: int = 1024,
                     seed: int = 0) -> GeometrySpec:
    """3D non-circular cone beam: saddle trajectory (phi = 5 deg cos 2 theta)
    with seeded per-view jitter (+-2 mm on x_src, z_src, u_ofst, v_ofst and
    +-0.5 deg on theta, phi, psi), n^3 volume of 0.4*512/n mm voxels, flat
    ndet x ndet detector of 0.4*1024/ndet mm, SAD 785 mm, SDD 1200 mm."""
    rng = np.random.default_rng(seed)
    th = _angles(nview)
    d2r = math.pi / 180.0
    jit = lambda w: rng.uniform(-w, w, nview)
    theta = th + jit(0.5 * d2r)
    phi = 5.0 * d2r * np.cos(2 * th) + jit(0.5 * d2r)
    psi = jit(0.5 * d2r)
    h = 0.4 * 512 / n
    dd = 0.4 * 1024 / ndet
    return GeometrySpec("noncirc3d", "flat", n, n, n, h, h, h,
                        ndet, ndet, dd, dd, nview, theta=theta, phi=phi, psi=psi,
                        sad=785.0, sdd=1200.0, x_src=jit(2.0), z_src=jit(2.0),
                        u_ofst=jit(2.0), v_ofst=jit(2.0))


def scaled(spec: GeometrySpec, n: int, nview: int, ndet_u: Optional[int] = None,
           ndet_v: Optional[int] = None) -> GeometrySpec:
    """A smaller copy of `spec` covering the same physical field of view:
    n voxels per transaxial side (nz scaled in proportion), nview views over
    the same angular span, detector cells enlarged in proportion."""
    kw = dataclasses.asdict(spec)
    fx = spec.nx / n
    kw["nx"], kw["ny"] = n, n
    kw["dx"], kw["dy"] = spec.dx * fx, spec.dy * fx
    if spec.kind != "fan2d":
        nz = max(1, int(round(spec.nz / fx)))
        kw["dz"] = spec.dz * spec.nz / nz
        kw["nz"] = nz
    nu = ndet_u or max(4, int(round(spec.nu / fx)))
    kw["du"] = spec.du * spec.nu / nu
    kw["nu"] = nu
    if spec.kind != "fan2d":
        nv = ndet_v or max(2, int(round(spec.nv / fx)))
        kw["dv"] = spec.dv * spec.nv / nv
        kw["nv"] = nv
    sel = np.round(np.arange(nview) * spec.nview / nview).astype(np.int64)
    kw["nview"] = nview
    for name in PER_VIEW:
        a = spec.param(name)
        kw[name] = a.copy() if a.size == 1 else a[sel].copy()
    if spec.poses is not None:
        kw["poses"] = np.asarray(spec.poses)[sel].copy()
    return GeometrySpec(**kw)


# -- phantoms --------------------------------------------------------------------

def ellipse_params(seed: int, ndim: int, count: Optional[int] = None):
    """Parameters of the random-ellipse/ellipsoid phantom, in units of the
    field-of-view half extent: (centre, semi-axes, rotation, value) per body.
    Centres uniform in 0.7 x half extent, semi-axes uniform in [0.05, 0.45] x
    extent, uniformly random orientation, value uniform in [0, 0.03] / mm."""
    rng = np.random.default_rng(seed)
    k = count if count is not None else (12 if ndim == 2 else 24)
    out = []
    for _ in range(k):
        c = rng.uniform(-0.7, 0.7, ndim)
        a = rng.uniform(0.05, 0.45, ndim) * 2.0
        if ndim == 2:
            t = rng.uniform(0, math.pi)
            rot = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
        else:
            q = rng.normal(size=4)
            q /= np.linalg.norm(q)
            w, x, y, z = q
            rot = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
        val = rng.uniform(0.0, 0.03)
        out.append((c, a, rot, val))
    return out


def phantom(spec: GeometrySpec, seed: int = 0, device=None, dtype=None):
    """Seeded random-ellipse (2D) or ellipsoid (3D) phantom sampled at voxel
    centres, shape (nz, ny, nx), values in [0, 0.03] / mm.  Bodies are drawn in
    order and later ones overwrite earlier ones.  Returns a float64 numpy array,
    or a torch tensor on `device` when one is given (computed there)."""
    ndim = 2 if spec.kind == "fan2d" else 3
    params = ellipse_params(seed, ndim)
    if device is None:
        return _phantom_numpy(spec, params, ndim)
    import torch
    return _phantom_torch(spec, params, ndim, torch.device(device),
                          dtype or torch.float32)


def _grid_coords(n, h):
    return (np.arange(n, dtype=np.float64) - (n - 1) / 2.0) * h


def _phantom_numpy(spec, params, ndim):
    nz, ny, nx = spec.vol_shape
    hx = spec.nx * spec.dx / 2.0
    hy = spec.ny * spec.dy / 2.0
    hz = spec.nz * spec.dz / 2.0
    xs = _grid_coords(nx, spec.dx) / hx
    ys = _grid_coords(ny, spec.dy) / hy
    zs = _grid_coords(nz, spec.dz) / hz if ndim == 3 else np.zeros(1)
    out = np.zeros((nz, ny, nx))
    for c, a, rot, val in params:
        # bounding box of the body (half extent along axis i: |R_i. * a|)
        ext = np.sqrt(((rot * a[None, :]) ** 2).sum(1))
        cz = c[2] if ndim == 3 else 0.0
        ez = ext[2] if ndim == 3 else 1.0
        ix = np.nonzero(np.abs(xs - c[0]) <= ext[0] + 1e-12)[0]
        iy = np.nonzero(np.abs(ys - c[1]) <= ext[1] + 1e-12)[0]
        iz = np.nonzero(np.abs(zs - cz) <= ez + 1e-12)[0] if ndim == 3 else np.zeros(1, int)
        if ix.size == 0 or iy.size == 0 or iz.size == 0:
            continue
        X = xs[ix][None, None, :] - c[0]
        Y = ys[iy][None, :, None] - c[1]
        if ndim == 2:
            p0 = X * rot[0, 0] + Y * rot[1, 0]
            p1 = X * rot[0, 1] + Y * rot[1, 1]
            m = (p0 / a[0]) ** 2 + (p1 / a[1]) ** 2 <= 1.0
        else:
            Z = zs[iz][:, None, None] - cz
            p0 = X * rot[0, 0] + Y * rot[1, 0] + Z * rot[2, 0]
            p1 = X * rot[0, 1] + Y * rot[1, 1] + Z * rot[2, 1]
            p2 = X * rot[0, 2] + Y * rot[1, 2] + Z * rot[2, 2]
            m = (p0 / a[0]) ** 2 + (p1 / a[1]) ** 2 + (p2 / a[2]) ** 2 <= 1.0
        sub = out[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1]
        sub[np.broadcast_to(m, sub.shape)] = val
    return out


def _phantom_torch(spec, params, ndim, device, dtype):
    import torch
    nz, ny, nx = spec.vol_shape
    f64 = torch.float64
    hx = spec.nx * spec.dx / 2.0
    hy = spec.ny * spec.dy / 2.0
    hz = spec.nz * spec.dz / 2.0
    xs = torch.as_tensor(_grid_coords(nx, spec.dx) / hx, dtype=f64, device=device)
    ys = torch.as_tensor(_grid_coords(ny, spec.dy) / hy, dtype=f64, device=device)
    zs = (torch.as_tensor(_grid_coords(nz, spec.dz) / hz, dtype=f64, device=device)
          if ndim == 3 else torch.zeros(1, dtype=f64, device=device))
    out = torch.zeros((nz, ny, nx), dtype=f64, device=device)
    for c, a, rot, val in params:
        cz = c[2] if ndim == 3 else 0.0
        X = (xs - c[0]).view(1, 1, -1)
        Y = (ys - c[1]).view(1, -1, 1)
        if ndim == 2:
            p0 = X * rot[0, 0] + Y * rot[1, 0]
            p1 = X * rot[0, 1] + Y * rot[1, 1]
            m = (p0 / a[0]) ** 2 + (p1 / a[1]) ** 2 <= 1.0
        else:
            Z = (zs - cz).view(-1, 1, 1)
            p0 = X * rot[0, 0] + Y * rot[1, 0] + Z * rot[2, 0]
            p1 = X * rot[0, 1] + Y * rot[1, 1] + Z * rot[2, 1]
            p2 = X * rot[0, 2] + Y * rot[1, 2] + Z * rot[2, 2]
            m = (p0 / a[0]) ** 2 + (p1 / a[1]) ** 2 + (p2 / a[2]) ** 2 <= 1.0
        out[m.expand(nz, ny, nx)] = val
    return out.to(dtype)


def random_volume(spec: GeometrySpec, seed: int = 0, batch: int = 1) -> np.ndarray:
    """Seeded U[0, 1) volume(s), shape (batch, nz, ny, nx), float64."""
    rng = np.random.default_rng(1000 + seed)
    return rng.random((batch,) + spec.vol_shape)


def random_sino(spec: GeometrySpec, seed: int = 0, batch: int = 1) -> np.ndarray:
    """Seeded U[0, 1) sinogram(s), shape (batch, nview, nv, nu), float64."""
    rng = np.random.default_rng(2000 + seed)
    return rng.random((batch,) + spec.sino_shape)
