"""Accumulating projections and the fused least-squares MBIR step
(Sec. 2.4) against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import workloads as W
from gpu_util import PROJECTORS, TOL_F32, ragged, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


@pytest.mark.parametrize("proj", PROJECTORS)
def test_accumulate_forms(ct, proj):
    spec = ragged("circ3d", "flat", seed=31)
    g = ct.Geometry.from_spec(spec)
    x0 = W.phantom(spec, seed=6)
    y0 = W.random_sino(spec, seed=6)[0]
    x = torch.as_tensor(x0, dtype=torch.float32).cuda()
    y = torch.as_tensor(y0, dtype=torch.float32).cuda()
    r = y.clone()
    ct.forward_acc(g, x, r, 2.0, -0.5, proj)
    assert rel_l2(r.cpu().numpy(), 2.0 * oracle.forward(spec, proj, x0) - 0.5 * y0) <= TOL_F32
    xb = x.clone()
    ct.back_acc(g, y, xb, -0.25, 3.0, proj)
    assert rel_l2(xb.cpu().numpy(), 3.0 * x0 - 0.25 * oracle.back(spec, proj, y0)) <= TOL_F32
    # alpha = 1, beta = 0 is the plain projection, bit for bit
    z = torch.full_like(y, 7.0)
    assert torch.equal(ct.forward_acc(g, x, z, 1.0, 0.0, proj), ct.forward(g, x, proj))


@pytest.mark.parametrize("proj", ["dd", "sf"])
def test_fused_ls_steps_match_oracle_iteration(ct, proj):
    from paper_2503_16741_gb300.mbir import ls_gradient_descent, ls_step_size
    spec = ragged("circ3d", "curved", seed=32)
    g = ct.Geometry.from_spec(spec)
    truth = W.phantom(spec, seed=7)
    y0 = oracle.forward(spec, proj, truth)
    lr = ls_step_size(g, proj)
    x = ls_gradient_descent(g, torch.as_tensor(y0, dtype=torch.float32).cuda(), proj, 3, lr=lr)
    xr = np.zeros_like(truth)
    for _ in range(3):
        xr = xr - lr * oracle.back(spec, proj, oracle.forward(spec, proj, xr) - y0)
    assert rel_l2(x.cpu().numpy(), xr) <= 3 * TOL_F32
    # the data term falls monotonically
    losses = []
    xk = torch.zeros_like(x)
    yd = torch.as_tensor(y0, dtype=torch.float32).cuda()
    for _ in range(6):
        losses.append(float(((ct.forward(g, xk, proj) - yd).double() ** 2).sum()))
        xk = ls_gradient_descent(g, yd, proj, 1, lr=lr, x0=xk)
    assert all(b < a for a, b in zip(losses, losses[1:])), losses


def test_ten_step_ls_loop_on_curved_geometry_matches_autograd(ct):
    """The 10-step least-squares loop (curved cone beam, DD): fused steps
    equal steps taken with torch.autograd through the Projector module."""
    from paper_2503_16741_gb300.mbir import ls_gradient_descent, ls_step_size
    spec = W.scaled(W.circ3d_curved(), 64, 123)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(W.phantom(spec, seed=8), dtype=torch.float32).cuda(), "dd")
    lr = ls_step_size(g, "dd")
    fused = ls_gradient_descent(g, y, "dd", 10, lr=lr)
    A = ct.Projector(g, "proj", "DD", "forward")
    x = torch.zeros_like(fused, requires_grad=True)
    for _ in range(10):
        loss = 0.5 * ((A(x) - y) ** 2).sum()
        (gr,) = torch.autograd.grad(loss, [x])
        x.data -= lr * gr
    assert rel_l2(fused.cpu().numpy(), x.detach().cpu().numpy()) <= 1e-5


@pytest.mark.parametrize("kind", ["circ3d", "noncirc3d"])
def test_geometry_subset_projects_those_rows(ct, kind):
    spec = ragged(kind, "flat", seed=40)
    g = ct.Geometry.from_spec(spec)
    x = torch.as_tensor(W.phantom(spec, seed=3), dtype=torch.float32).cuda()
    views = [2, 9, 10, 21]
    for proj in ("sf", "dd", "voxel", "ray"):
        assert torch.equal(ct.forward(g.subset(views), x, proj), ct.forward(g, x, proj)[views])


def test_one_ordered_subset_is_the_full_gradient_step(ct):
    from paper_2503_16741_gb300.mbir import ls_gradient_descent, ls_step_size, os_gradient_descent
    spec = ragged("circ3d", "flat", seed=41)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(W.phantom(spec, seed=4), dtype=torch.float32).cuda(), "sf")
    lr = ls_step_size(g, "sf")
    assert torch.equal(os_gradient_descent(g, y, "sf", 1, 3, lr=[lr]), ls_gradient_descent(g, y, "sf", 3, lr=lr))


@pytest.mark.parametrize("proj", ["sf", "dd"])
def test_ordered_subsets_match_oracle_iteration(ct, proj):
    """Two epochs over 3 interleaved view subsets: each step
    x <- x - lr_s A_s^T (A_s x - y_s) against the same iteration in FP64."""
    from paper_2503_16741_gb300.mbir import ls_step_size, ordered_subsets, os_gradient_descent
    spec = ragged("noncirc3d", "flat", seed=42)
    g = ct.Geometry.from_spec(spec)
    truth = W.phantom(spec, seed=5)
    y0 = oracle.forward(spec, proj, truth)
    subsets = ordered_subsets(spec.nview, 3)
    lrs = [ls_step_size(g.subset(v), proj) for v in subsets]
    x = os_gradient_descent(g, torch.as_tensor(y0, dtype=torch.float32).cuda(), proj, 3, 2, lr=lrs)
    xr = np.zeros_like(truth)
    for _ in range(2):
        for v, lr in zip(subsets, lrs):
            sub = spec.subset(v)
            xr = xr - lr * oracle.back(sub, proj, oracle.forward(sub, proj, xr) - y0[v])
    assert rel_l2(x.cpu().numpy(), xr) <= 3 * TOL_F32


def test_ordered_subsets_reduce_the_data_term_faster_per_epoch(ct):
    """An epoch over 6 subsets costs about one full gradient step (every view
    projected once each way) and lowers the data term further."""
    from paper_2503_16741_gb300.mbir import ls_gradient_descent, os_gradient_descent
    spec = ragged("circ3d", "flat", seed=43)
    g = ct.Geometry.from_spec(spec)
    y = ct.forward(g, torch.as_tensor(W.phantom(spec, seed=6), dtype=torch.float32).cuda(), "dd")
    loss = lambda x: float(((ct.forward(g, x, "dd") - y).double() ** 2).sum())
    full = ls_gradient_descent(g, y, "dd", 2)
    osx = os_gradient_descent(g, y, "dd", 6, 2)
    assert loss(osx) < loss(full) < loss(torch.zeros_like(full))
