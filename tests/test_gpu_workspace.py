"""ct_workspace_bytes against what the library's pool actually hands out:
for every projector, direction and geometry kind, the high-water mark of the
pool's bytes in use during one call equals the size the query reports (up
to the pool's allocation granularity), and is zero where the query says the
call takes no workspace."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from gpu_util import ragged

pytestmark = pytest.mark.gpu
GRANULE = 2 << 20  # the pool may round an allocation up to its page size


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def _specs():
    # nz a multiple of 4 (the streaming forwards' z-major copy) and ragged ones
    circ = W.scaled(W.circ3d_256(), 32, 20)
    return {"fan2d": ragged("fan2d", "flat", 5), "circ-flat": circ, "circ-curved": ragged("circ3d", "curved", 6),
            "circ-ragged": ragged("circ3d", "flat", 7), "noncirc": ragged("noncirc3d", "flat", 8)}


CASES = [(name, proj, d, dt) for name in _specs() for proj in ("voxel", "ray", "dd", "sf", "sftt")
         for d in ("fwd", "back") for dt in ("f32", "f16")
         if not (proj == "sftt" and name == "circ-curved")]
T = {"f32": torch.float32, "f16": torch.float16}


@pytest.mark.parametrize("name,proj,direction,dt", CASES, ids=["-".join(c) for c in CASES])
@pytest.mark.parametrize("batch", [1, 2])
def test_workspace_query_matches_the_pool(ct, name, proj, direction, dt, batch):
    spec = _specs()[name]
    g = ct.Geometry.from_spec(spec)
    want = ct.workspace_bytes(g, proj, direction, T[dt], batch)
    vol = (batch,) + g.vol_shape
    sino = (batch,) + g.sino_shape
    x = torch.rand(vol if direction == "fwd" else sino, device="cuda").to(T[dt])
    torch.cuda.synchronize()
    ct.workspace_usage(reset_high=True)
    out = ct.forward(g, x, proj) if direction == "fwd" else ct.back(g, x, proj)
    torch.cuda.synchronize()
    _, high = ct.workspace_usage()
    del out
    if want == 0:
        assert high == 0
    else:
        assert want <= high <= want + GRANULE, (want, high)


def test_workspace_limit_releases_freed_blocks(ct):
    """After a call with a large workspace, a limit of zero hands the pool's
    freed blocks back to the device."""
    spec = W.scaled(W.circ3d_256(), 64, 45)
    g = ct.Geometry.from_spec(spec)
    y = torch.rand(g.sino_shape, device="cuda")
    ct.workspace_limit(1 << 62)
    ct.back(g, y, "dd")
    torch.cuda.synchronize()
    held, _ = ct.workspace_usage()
    assert held >= ct.workspace_bytes(g, "dd", "back")
    ct.workspace_limit(0)
    held, _ = ct.workspace_usage()
    assert held == 0
    ct.workspace_limit(1 << 62)
