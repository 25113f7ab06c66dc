"""Differentiation (Sec. 2.1, Sec. 2.3: the projector and backprojector are
each other's gradient) and the MBIR example of Sec. 2.4."""
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
def test_gradient_of_least_squares_matches_oracle(ct, proj):
    """L(x) = 1/2 ||A x - y||^2 (sum form): grad = A^T (A x - y)."""
    spec = ragged("circ3d", "curved", seed=11)
    g = ct.Geometry.from_spec(spec)
    x0 = W.phantom(spec, seed=5)
    y = W.random_sino(spec, seed=5)[0] * 0.5
    x = torch.tensor(x0, dtype=torch.float32, device="cuda", requires_grad=True)
    yd = torch.as_tensor(y, dtype=torch.float32).cuda()
    A = ct.Projector(g, "proj", proj, "forward")
    loss = 0.5 * ((A(x) - yd) ** 2).sum()
    (grad,) = torch.autograd.grad(loss, [x])
    ref = oracle.back(spec, proj, oracle.forward(spec, proj, x0) - y)
    assert rel_l2(grad.cpu().numpy(), ref) <= TOL_F32


@pytest.mark.parametrize("proj", PROJECTORS)
def test_directional_finite_difference(ct, proj):
    """Central difference of the FP64-accumulated loss along a random
    direction agrees with <grad, d> to 1e-3 (FP32 forward evaluations)."""
    spec = ragged("noncirc3d", "flat", seed=12)
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(3)
    x = torch.rand(spec.vol_shape, generator=gen, device="cuda", requires_grad=True)
    y = torch.rand(spec.sino_shape, generator=gen, device="cuda")
    d = torch.randn(spec.vol_shape, generator=gen, device="cuda")
    A = ct.Projector(g, "proj", proj, "forward")

    def loss(v):
        r = (A(v) - y).double()
        return 0.5 * (r * r).sum()

    (grad,) = torch.autograd.grad(loss(x), [x])
    h = 1e-2
    with torch.no_grad():
        fd = (loss(x + h * d) - loss(x - h * d)) / (2 * h)
    an = (grad.double() * d.double()).sum()
    assert abs(float(fd - an)) <= 1e-3 * abs(float(an))


def test_backward_direction_module(ct):
    """direction='backward' is the adjoint; its gradient is the forward."""
    spec = ragged("fan2d", "flat", seed=13)
    g = ct.Geometry.from_spec(spec)
    gen = torch.Generator(device="cuda").manual_seed(4)
    s = torch.rand((spec.nview, spec.nu), generator=gen, device="cuda", requires_grad=True)
    w = torch.rand((spec.ny, spec.nx), generator=gen, device="cuda")
    At = ct.Projector(g, "proj", "dd", "backward")
    (gs,) = torch.autograd.grad((At(s) * w).sum(), [s])
    assert torch.allclose(gs, ct.forward(g, w.contiguous(), "dd"))


def test_mbir_gradient_descent_reduces_the_data_term(ct):
    """The example of Sec. 2.4: x <- x - lr * grad of mse_loss(A(x), sino),
    with lr = 1 / L, L = 2 ||A||^2 / N the gradient's Lipschitz constant
    (||A||^2 from a power iteration on A^T A): the loss must fall monotonically."""
    spec = W.scaled(W.fan2d_small(), 64, 90)
    g = ct.Geometry.from_spec(spec)
    img = torch.as_tensor(W.phantom(spec, seed=1)[0], dtype=torch.float32).cuda()
    A = ct.Projector(g, "proj", "sf", "forward")
    sino = A(img[None, None]).detach()
    v = torch.rand_like(img)
    for _ in range(20):
        v = ct.back(g, ct.forward(g, v, "sf"), "sf")
        nrm = v.norm()
        v = v / nrm
    L = 2.0 * float(nrm) / sino.numel()
    x = torch.zeros_like(img[None, None], requires_grad=True)
    losses = []
    for _ in range(10):
        loss = torch.nn.functional.mse_loss(A(x), sino)
        (grad,) = torch.autograd.grad(loss, [x])
        x.data -= grad / L
        losses.append(float(loss.detach()))
    assert all(b < a for a, b in zip(losses, losses[1:])), losses
    assert losses[-1] < 0.5 * losses[0], losses


def test_projector_module_recon_mode(ct):
    """Projector(mode='recon', direction='backward') is the FBP
    backprojection of filtered projections (ct_back in CT_MODE_RECON)."""
    from paper_2503_16741_gb300.autograd import Projector
    spec = W.scaled(W.circ3d_256(), 32, 40)
    g = ct.Geometry.from_spec(spec)
    y = torch.rand(g.sino_shape, device="cuda")
    q = ct.ramp_filter(g, y)
    for method in ("voxel", "DD", "SF"):
        got = Projector(g, "recon", method, "backward")(q)
        ref = ct.back(g, q, method.lower(), mode="recon")
        torch.cuda.synchronize()
        assert torch.equal(got, ref)
    with pytest.raises(ValueError):
        Projector(g, "recon", "SF", "forward")
