"""Helpers for the GPU parity tests: geometries that span several kernel
tiles with ragged edges, and the error measure used throughout."""
import numpy as np

import workloads as W

# relative L2 bound of the FP32 path against the FP64 oracle
TOL_F32 = 1e-5
# relative L2 bound of FP16 storage (FP32 arithmetic) against the FP64 oracle
TOL_F16 = 1e-3


def rel_l2(got, ref) -> float:
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def ragged(kind: str, det: str, seed: int = 0) -> W.GeometrySpec:
    """Small geometries whose sizes are not multiples of the 32x8 / 32x4
    thread tiles, with every offset of Sec. 2.2 set, and a detector that
    truncates part of the volume."""
    rng = np.random.default_rng(100 + seed)
    nview = 23
    theta = np.sort(rng.uniform(0, 2 * np.pi, nview))
    if kind == "fan2d":
        return W.GeometrySpec("fan2d", det, 45, 38, 1, 1.7, 1.7, 1.0, 70, 1, 1.9, 1.0, nview,
                              theta=theta, sad=300.0, sdd=620.0, x_src=1.5, u_ofst=2.3,
                              x_ofst=-3.0, y_ofst=2.0)
    kw = dict(theta=theta, sad=320.0, sdd=640.0, x_src=1.2, z_src=-2.0, u_ofst=-2.6,
              v_ofst=1.7, x_ofst=2.0, y_ofst=-1.0, z_ofst=1.5)
    if kind == "noncirc3d":
        kw["phi"] = np.deg2rad(5.0) * np.cos(2 * theta) + rng.uniform(-0.01, 0.01, nview)
        kw["psi"] = rng.uniform(-0.01, 0.01, nview)
        kw["x_src"] = 1.2 + rng.uniform(-2, 2, nview)
    return W.GeometrySpec(kind, det, 37, 34, 21, 1.6, 1.6, 1.3, 61, 29, 2.2, 2.1, nview, **kw)


GEOMS = [("fan2d", "flat"), ("fan2d", "curved"), ("circ3d", "flat"), ("circ3d", "curved"),
         ("noncirc3d", "flat")]
PROJECTORS = ["voxel", "ray", "dd", "sf"]
