"""Brute-force NumPy references used to pin the oracle.

Every (ray, voxel) pair is tested with the slab method, with no candidate
pruning and no incremental traversal, so an error in the oracle's Siddon walk
or in its candidate-cell enumeration shows up as a mismatch.  Ray end points
(source and cell centres) come from the oracle's geometry, which is pinned
separately against hand-derived frames in test_oracle_geometry.py.
"""
import numpy as np

import oracle


def voxel_boxes(spec, view=0):
    """Half-open boxes [lo, hi) of every voxel, flat order (k, j, i)."""
    nz = 1 if spec.kind == "fan2d" else spec.nz
    dz = 1.0 if spec.kind == "fan2d" else spec.dz
    xo = spec.per_view("x_ofst")[view]
    yo = spec.per_view("y_ofst")[view]
    zo = 0.0 if spec.kind == "fan2d" else spec.per_view("z_ofst")[view]
    xc = (np.arange(spec.nx) - (spec.nx - 1) / 2) * spec.dx + xo
    yc = (np.arange(spec.ny) - (spec.ny - 1) / 2) * spec.dy + yo
    zc = (np.arange(nz) - (nz - 1) / 2) * dz + zo
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    ctr = np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)
    h = np.array([spec.dx, spec.dy, dz]) / 2
    return ctr - h, ctr + h


def seg_lengths(s, P, lo, hi):
    """Length of segment s -> P inside each half-open box; s, P: (3,) or (R, 3);
    lo, hi: (N, 3).  Returns (N,) or (R, N)."""
    s = np.atleast_2d(s)[:, None, :]
    P = np.atleast_2d(P)[:, None, :]
    d = P - s
    lo = lo[None]
    hi = hi[None]
    t0 = np.zeros(np.broadcast_shapes(d.shape, lo.shape)[:2])
    t1 = np.ones_like(t0)
    for m in range(3):
        dm = d[..., m]
        zero = dm == 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (lo[..., m] - s[..., m]) / dm
            tb = (hi[..., m] - s[..., m]) / dm
        inside = (s[..., m] >= lo[..., m]) & (s[..., m] < hi[..., m])
        lo_t = np.where(zero, np.where(inside, -np.inf, np.inf), np.minimum(ta, tb))
        hi_t = np.where(zero, np.where(inside, np.inf, -np.inf), np.maximum(ta, tb))
        t0 = np.maximum(t0, lo_t)
        t1 = np.minimum(t1, hi_t)
    L = np.linalg.norm(d, axis=-1)
    out = np.where(t1 > t0, (t1 - t0) * L, 0.0)
    return out[0] if out.shape[0] == 1 else out


def ray_system_matrix(spec):
    """Dense ray-driven system matrix, rows (view, b, a), columns (k, j, i)."""
    nv = 1 if spec.kind == "fan2d" else spec.nv
    nz = 1 if spec.kind == "fan2d" else spec.nz
    A = np.zeros((spec.nview * nv * spec.nu, spec.nx * spec.ny * nz))
    r = 0
    for v in range(spec.nview):
        lo, hi = voxel_boxes(spec, v)
        s = oracle.frame(spec, v)["s"]
        for b in range(nv):
            P = np.array([oracle.cell_point(spec, v, a, b) for a in range(spec.nu)])
            A[r:r + spec.nu] = seg_lengths(s, P, lo, hi)
            r += spec.nu
    return A


def subray_average_parallel_2d(spec, image, view, nsub):
    """Cell-averaged exact parallel-beam line integrals of a 2D pixel image:
    each cell is sampled by `nsub` rays parallel to the detector normal, at
    the midpoints of equal sub-intervals of the cell (midpoint rule).  This is
    the limit that a divergent geometry with very large SAD and SDD emulates
    (Sec. 2.2)."""
    f = oracle.frame(spec, view)
    lo, hi = voxel_boxes(spec, view)
    x = image.ravel()
    out = np.zeros(spec.nu)
    offs = ((np.arange(nsub) + 0.5) / nsub - 0.5) * spec.du
    reach = 4.0 * (spec.nx * spec.dx + spec.ny * spec.dy)
    for a in range(spec.nu):
        ua = (a - (spec.nu - 1) / 2) * spec.du
        # detector points pulled back to a plane through the rotation centre
        P = (ua + offs)[:, None] * f["eu"][None] + 0.5 * reach * f["n"][None]
        S = P - reach * f["n"][None]
        acc = 0.0
        for c0 in range(0, nsub, 512):
            L = seg_lengths(S[c0:c0 + 512], P[c0:c0 + 512], lo, hi)
            acc += (np.atleast_2d(L) @ x).sum()
        out[a] = acc / nsub
    return out
