"""PyTorch autograd integration (Sec. 2.1): the forward projector and the
backprojector are each other's gradient (Sec. 2.3: grad_x (A x) = A^T,
grad_y (A^T y) = A), so each direction's backward calls the other kernel."""
from __future__ import annotations

import torch

from .binding import Geometry, back, forward


class ProjectorFn(torch.autograd.Function):
    """y = A x for direction 'forward', x = A^T y for 'backward'."""

    @staticmethod
    def forward(ctx, inp: torch.Tensor, geom: Geometry, projector: str, direction: str):
        ctx.geom, ctx.projector, ctx.direction = geom, projector, direction
        inp = inp.contiguous()
        if direction == "forward":
            return forward(geom, inp, projector)
        return back(geom, inp, projector)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = grad_out.contiguous()
        if ctx.direction == "forward":
            grad_in = back(ctx.geom, g, ctx.projector)
        else:
            grad_in = forward(ctx.geom, g, ctx.projector)
        return grad_in, None, None, None


class Projector(torch.nn.Module):
    """Projector(geom, mode, method, direction) -- the unified projector
    module of Sec. 2.1 / Sec. 2.4: method in {'voxel', 'ray', 'DD', 'SF'}
    (and 'SFTT'), direction 'forward' (volume -> sinogram) or 'backward'.
    mode 'proj': the matched pair, each direction the other's gradient.
    mode 'recon' (Sec. 2.3): the backward direction is the depth-weighted FBP
    backprojection of ramp-filtered projections (voxel-driven, DD or SF
    interpolation).  Its own adjoint is not the forward projector, and the
    library provides no recon-mode forward, so it runs without autograd."""

    def __init__(self, geom: Geometry, mode: str = "proj", method: str = "SF",
                 direction: str = "forward"):
        super().__init__()
        if mode not in ("proj", "recon"):
            raise ValueError("mode must be 'proj' or 'recon'")
        if direction not in ("forward", "backward"):
            raise ValueError("direction must be 'forward' or 'backward'")
        if mode == "recon" and direction != "backward":
            raise ValueError("recon mode is a backprojection: direction must be 'backward'")
        self.geom = geom
        self.mode = mode
        self.method = method.lower()
        self.direction = direction

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        if self.mode == "recon":
            with torch.no_grad():
                return back(self.geom, x.detach().contiguous(), self.method, mode="recon")
        return ProjectorFn.apply(x, self.geom, self.method, self.direction)
