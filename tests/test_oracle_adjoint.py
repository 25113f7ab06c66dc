"""The oracle's forward and back projections are a matched pair (Sec. 2.3,
Eq. 1-2): <A x, y> = <x, A^T y> to FP64 rounding, for every projector and
geometry.  For the ray-driven projector the two sides are computed by
different algorithms (Siddon walk forward, per-voxel slab test backward), so
this also pins one against the other."""
import numpy as np
import pytest

import oracle
import workloads as W

GEOMS = {
    "fan2d-flat": W.GeometrySpec("fan2d", "flat", 24, 20, 1, 1.5, 1.5, 1.0, 48, 1, 1.3, 1.0, 11,
                                 theta=np.linspace(0, 6.2, 11), sad=200.0, sdd=420.0,
                                 x_src=1.0, u_ofst=-0.7, x_ofst=2.0, y_ofst=-1.5),
    "fan2d-curved": W.GeometrySpec("fan2d", "curved", 24, 20, 1, 1.5, 1.5, 1.0, 48, 1, 1.3, 1.0, 11,
                                   theta=np.linspace(0, 6.2, 11), sad=200.0, sdd=420.0,
                                   u_ofst=1.625),
    "circ3d-flat": W.scaled(W.circ3d_256(), 14, 9),
    "circ3d-curved": W.scaled(W.circ3d_curved(), 16, 9),
    "noncirc3d": W.scaled(W.noncirc3d_saddle(), 12, 9),
}


@pytest.mark.parametrize("proj", ["voxel", "ray", "dd", "sf"])
@pytest.mark.parametrize("name", sorted(GEOMS))
def test_adjoint_identity(name, proj):
    spec = GEOMS[name]
    x = W.random_volume(spec, 11, batch=2)
    y = W.random_sino(spec, 11, batch=2)
    Ax = oracle.forward(spec, proj, x)
    Aty = oracle.back(spec, proj, y)
    for b in range(2):
        lhs = np.vdot(Ax[b], y[b])
        rhs = np.vdot(x[b], Aty[b])
        assert lhs > 0
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("proj", ["voxel", "ray", "dd", "sf"])
def test_batch_items_are_independent(proj):
    spec = GEOMS["circ3d-flat"]
    x = W.random_volume(spec, 12, batch=3)
    Ax = oracle.forward(spec, proj, x)
    for b in range(3):
        np.testing.assert_array_equal(Ax[b], oracle.forward(spec, proj, x[b]))


@pytest.mark.parametrize("proj", ["voxel", "ray", "dd", "sf"])
def test_back_voxels_matches_full_back(proj):
    spec = GEOMS["noncirc3d"]
    y = W.random_sino(spec, 13)[0]
    full = oracle.back(spec, proj, y).ravel()
    sel = np.array([0, 5, 77, 300, spec.n_vox - 1])
    np.testing.assert_allclose(oracle.back_voxels(spec, proj, y, sel), full[sel], rtol=1e-14)


@pytest.mark.parametrize("proj", ["voxel", "ray", "dd", "sf"])
def test_view_subset_is_the_restricted_operator(proj):
    """Per-view geometry (Sec. 2.2) makes a view subset a geometry of its own:
    the forward of the subset equals those views of the full forward."""
    spec = GEOMS["noncirc3d"]
    x = W.random_volume(spec, 14)[0]
    full = oracle.forward(spec, proj, x)
    views = [1, 4, 8]
    np.testing.assert_array_equal(oracle.forward(spec.subset(views), proj, x), full[views])
