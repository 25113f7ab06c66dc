"""Model-based iterative reconstruction by gradient descent on the
least-squares data term (the example of Sec. 2.4, Eq. 3 without the TV term):
x <- x - lr * A^T (A x - y), over all views or over ordered subsets of them.

Each step is two library calls on one stream: ct_forward_acc forms the
residual r = A x - y in place of a copy of y, and ct_back_acc applies
x <- x - lr A^T r in place -- no elementwise passes and no host round trip.
Ordered subsets (OS) take the step with the views of one subset at a time
(A_s, y_s: the subset's rows), cycling through the subsets; each subset is a
geometry of its own (Geometry.subset).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import torch

from .binding import Geometry, back, back_acc, forward, forward_acc


def operator_norm_sq(geom: Geometry, projector: str, iters: int = 12, batch_shape=(),
                     stream=None, seed: int = 0) -> float:
    """||A||_2^2 (largest eigenvalue of A^T A) by power iteration."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    v = torch.rand(tuple(batch_shape) + geom.vol_shape, generator=gen, device="cuda")
    lam = 0.0
    for _ in range(iters):
        w = back(geom, forward(geom, v, projector, stream=stream), projector, stream=stream)
        lam = float(w.norm())
        v = w / max(lam, 1e-30)
    return lam


def ls_step_size(geom: Geometry, projector: str, **kw) -> float:
    """1 / ||A||^2: the step that makes x <- x - lr A^T (A x - y) monotone in
    1/2 ||A x - y||^2 (with a 2% margin on the power-iteration estimate)."""
    return 1.0 / (1.02 * operator_norm_sq(geom, projector, **kw))


def ls_gradient_descent(geom: Geometry, y: torch.Tensor, projector: str, steps: int,
                        lr: Optional[float] = None, x0: Optional[torch.Tensor] = None,
                        stream=None, work: Optional[torch.Tensor] = None) -> torch.Tensor:
    """`steps` gradient steps on 1/2 ||A x - y||^2 from x0 (zeros by default).
    y: (..., nview, [nv,] nu); returns x with y's batch shape and dtype.  The
    residual A x - y is kept in FP32 whatever y's storage type (in half
    storage the difference of two close values would lose its digits)."""
    if lr is None:
        lr = ls_step_size(geom, projector)
    lead = y.shape[:-len(geom.sino_shape)]
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        x = (torch.zeros(tuple(lead) + geom.vol_shape, dtype=y.dtype, device=y.device)
             if x0 is None else x0.clone())
        r = torch.empty(y.shape, dtype=torch.float32, device=y.device) if work is None else work
        for _ in range(steps):
            r.copy_(y)
            forward_acc(geom, x, r, 1.0, -1.0, projector, stream=s)
            back_acc(geom, r, x, -lr, 1.0, projector, stream=s)
    return x


def ordered_subsets(nview: int, n_subsets: int) -> List[List[int]]:
    """Interleaved view subsets: subset s holds views s, s + S, s + 2S, ...
    (every view once; consecutive subsets are spread over the whole arc)."""
    if not 1 <= n_subsets <= nview:
        raise ValueError("need 1 <= n_subsets <= nview")
    return [list(range(s, nview, n_subsets)) for s in range(n_subsets)]


def os_gradient_descent(geom: Geometry, y: torch.Tensor, projector: str, n_subsets: int, epochs: int,
                        lr: Optional[Sequence[float]] = None, x0: Optional[torch.Tensor] = None,
                        stream=None, subsets: Optional[List[List[int]]] = None) -> torch.Tensor:
    """`epochs` passes over the ordered subsets, one gradient step on
    1/2 ||A_s x - y_s||^2 per subset s, with step lr[s] (default
    1 / ||A_s||^2 with the same 2 % margin as ls_step_size).
    y: (..., nview, [nv,] nu); returns x with y's batch shape and dtype
    (residuals in FP32)."""
    subsets = subsets if subsets is not None else ordered_subsets(geom.nview, n_subsets)
    geoms = [geom.subset(v) for v in subsets]
    if lr is None:
        lr = [ls_step_size(g, projector) for g in geoms]
    k = len(geom.sino_shape)
    lead = y.shape[:-k]
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        idx = [torch.as_tensor(v, device=y.device) for v in subsets]
        ys = [y.index_select(y.dim() - k, i).contiguous() for i in idx]
        rs = [torch.empty(t.shape, dtype=torch.float32, device=t.device) for t in ys]
        x = (torch.zeros(tuple(lead) + geom.vol_shape, dtype=y.dtype, device=y.device)
             if x0 is None else x0.clone())
        for _ in range(epochs):
            for g, ysub, r, step in zip(geoms, ys, rs, lr):
                r.copy_(ysub)
                forward_acc(g, x, r, 1.0, -1.0, projector, stream=s)
                back_acc(g, r, x, -step, 1.0, projector, stream=s)
    return x


def total_variation(x: torch.Tensor, eps: float = 1e-4) -> torch.Tensor:
    """Smoothed isotropic total variation of the last three (or two) axes:
    sum sqrt(|forward differences|^2 + eps^2), zero difference past the last
    voxel.  Written with torch operations, so autograd differentiates it."""
    nd = 3 if x.dim() >= 3 else 2
    sq = torch.zeros_like(x)
    for ax in range(x.dim() - nd, x.dim()):
        d = torch.diff(x, dim=ax, append=x.narrow(ax, x.shape[ax] - 1, 1))
        sq = sq + d * d
    return torch.sqrt(sq + eps * eps).sum()


def tv_mbir_adam(geom: Geometry, y: torch.Tensor, projector: str, iters: int, lam: float, lr: float,
                 x0: Optional[torch.Tensor] = None, eps: float = 1e-4):
    """MBIR with the objective of Sec. 3 (Eq. 3): ||A x - y||^2 + lam TV(x),
    minimised by `iters` Adam steps whose gradient comes from autograd through
    the projector (the forward's backward is the library's backprojection).
    Returns (x, objective after each step)."""
    from .autograd import Projector
    A = Projector(geom, "proj", projector, "forward")
    x = (torch.zeros(geom.vol_shape, dtype=torch.float32, device=y.device) if x0 is None
         else x0.detach().clone().float())
    x.requires_grad_(True)
    opt = torch.optim.Adam([x], lr=lr)
    history = []
    for _ in range(iters):
        opt.zero_grad(set_to_none=True)
        r = A(x) - y
        loss = (r * r).sum()
        if lam > 0:
            loss = loss + lam * total_variation(x, eps)
        loss.backward()
        opt.step()
        history.append(loss.detach())
    return x.detach(), torch.stack(history).cpu().tolist()
