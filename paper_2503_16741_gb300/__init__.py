"""GB300 CT projectors: forward projection y = A x and its matched adjoint
x = A^T y for fan-beam, circular and non-circular cone-beam geometries with
flat or curved detectors, with voxel-driven, ray-driven, distance-driven and
separable-footprint weights (CTorch, arXiv 2503.16741, Sec. 2).

All projection work runs in hand-written sm_103a kernels behind the C ABI of
include/ctproj.h; this package marshals PyTorch tensors to it.
"""
from .autograd import Projector, ProjectorFn
from .binding import (CTError, Geometry, back, back_acc, back_dd_noalloc, back_into, fbp, forward,
                      forward_acc, forward_into, lib_path, load, ramp_filter, workspace_bytes, workspace_limit,
                      workspace_usage)

__all__ = ["Geometry", "forward", "back", "forward_into", "back_into", "forward_acc", "back_acc",
           "back_dd_noalloc", "ramp_filter", "fbp", "workspace_bytes", "workspace_limit", "workspace_usage",
           "ProjectorFn", "Projector", "CTError", "load", "lib_path"]
