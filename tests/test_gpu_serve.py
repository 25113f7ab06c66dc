"""The continuous-batching server on the GPU: mixed requests arriving
together are batched and overlapped, and each result equals the same request
run alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from gpu_util import ragged

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ct():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2503_16741_gb300 as ct
    ct.load()
    return ct


def gdict(spec):
    return dict(kind=spec.kind, det=spec.det, nx=spec.nx, ny=spec.ny, nz=spec.nz, dx=spec.dx,
                dy=spec.dy, dz=spec.dz, nu=spec.nu, nv=spec.nv, du=spec.du, dv=spec.dv,
                nview=spec.nview, theta=spec.theta, phi=spec.phi, psi=spec.psi, sad=spec.sad,
                sdd=spec.sdd, x_src=spec.x_src, z_src=spec.z_src, x_ofst=spec.x_ofst,
                y_ofst=spec.y_ofst, z_ofst=spec.z_ofst, u_ofst=spec.u_ofst, v_ofst=spec.v_ofst)


def test_results_alone_equal_results_in_the_mix(ct):
    from paper_2503_16741_gb300.mbir import ls_gradient_descent
    from paper_2503_16741_gb300.serve import Request, Server
    specs = [ragged("fan2d", "flat", 41), ragged("circ3d", "flat", 42), ragged("circ3d", "curved", 43),
             ragged("noncirc3d", "flat", 44)]
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(32):
        sp = specs[k % 4]
        op = ["fwd", "back", "mbir", "fbp"][k % 4 if k >= 24 else k % 3]
        proj = ["sf", "dd", "voxel", "ray"][(k // 3) % 4]
        vol = (sp.ny, sp.nx) if sp.kind == "fan2d" else sp.vol_shape
        sino = (sp.nview, sp.nu) if sp.kind == "fan2d" else sp.sino_shape
        data = rng.random(vol if op == "fwd" else sino).astype(np.float32)
        reqs.append(Request(gdict(sp), op, data, projector=proj, iters=3))
    srv = Server(device=0, slots=4, hbm_budget=1 << 30, max_batch=4)
    futs = [srv.submit(r) for r in reqs]
    outs = [f.result(timeout=120) for f in futs]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs)
    assert st["launches"] <= len(reqs)
    for r, out in zip(reqs, outs):
        g = srv.ex.geometry(r.geometry)
        d = torch.as_tensor(r.data).cuda()
        if r.op == "fwd":
            alone = ct.forward(g, d, r.projector)
        elif r.op == "back":
            alone = ct.back(g, d, r.projector)
        elif r.op == "fbp":
            alone = ct.fbp(g, d)
        else:
            lr = srv.ex.step_size(r.geometry, r.projector)
            alone = ls_gradient_descent(g, d, r.projector, r.iters, lr=lr)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out, alone.cpu().numpy())


def test_server_rejects_requests_above_the_budget(ct):
    from paper_2503_16741_gb300.serve import Request, Server
    sp = W.scaled(W.circ3d_256(), 64, 90)
    srv = Server(device=0, slots=2, hbm_budget=1 << 20)
    fut = srv.submit(Request(gdict(sp), "fwd", np.zeros(sp.vol_shape, np.float32)))
    with pytest.raises(MemoryError):
        fut.result(timeout=30)
    srv.close()
