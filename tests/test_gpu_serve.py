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


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_half_storage_results_alone_equal_results_in_the_mix(ct, dtype):
    """The same alone-versus-mix equality in half storage (FP16 / BF16
    volumes and sinograms; MBIR keeps its residual in FP32)."""
    from paper_2503_16741_gb300.mbir import ls_gradient_descent
    from paper_2503_16741_gb300.serve import Request, Server
    T = {"f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    specs = [ragged("fan2d", "flat", 51), ragged("circ3d", "flat", 52), ragged("circ3d", "curved", 53),
             ragged("noncirc3d", "flat", 54)]
    rng = np.random.default_rng(1)
    reqs = []
    for k in range(24):
        sp = specs[k % 4]
        op = ["fwd", "back", "mbir"][k % 3]
        proj = ["sf", "dd"][(k // 3) % 2]
        vol = (sp.ny, sp.nx) if sp.kind == "fan2d" else sp.vol_shape
        sino = (sp.nview, sp.nu) if sp.kind == "fan2d" else sp.sino_shape
        data = rng.random(vol if op == "fwd" else sino).astype(np.float32)
        reqs.append(Request(gdict(sp), op, data, projector=proj, iters=3, dtype=dtype))
    srv = Server(device=0, slots=4, hbm_budget=1 << 30, max_batch=4)
    outs = [f.result(timeout=120) for f in [srv.submit(r) for r in reqs]]
    srv.close()
    for r, out in zip(reqs, outs):
        g = srv.ex.geometry(r.geometry)
        d = torch.as_tensor(r.data).cuda().to(T)
        if r.op == "fwd":
            alone = ct.forward(g, d, r.projector)
        elif r.op == "back":
            alone = ct.back(g, d, r.projector)
        else:
            lr = srv.ex.step_size(r.geometry, r.projector)
            alone = ls_gradient_descent(g, d, r.projector, r.iters, lr=lr)
        torch.cuda.synchronize()
        assert alone.dtype == T
        np.testing.assert_array_equal(out, alone.float().cpu().numpy())


def test_device_resident_requests(ct):
    """Requests that carry device tensors and ask for device results give
    what host requests give, and their inputs are used in place."""
    from paper_2503_16741_gb300.serve import Request, Server
    sp = ragged("circ3d", "flat", 61)
    rng = np.random.default_rng(2)
    host, dev = [], []
    for k in range(8):
        op = ["fwd", "back"][k % 2]
        data = rng.random(sp.vol_shape if op == "fwd" else sp.sino_shape).astype(np.float32)
        host.append(Request(gdict(sp), op, data, projector="sf"))
        dev.append(Request(gdict(sp), op, torch.as_tensor(data, device="cuda"), projector="sf", out_device=True))
    srv = Server(device=0, slots=3, hbm_budget=1 << 30, max_batch=3)
    fh = [srv.submit(r) for r in host]
    fd = [srv.submit(r) for r in dev]
    oh = [f.result(timeout=60) for f in fh]
    od = [f.result(timeout=60) for f in fd]
    srv.close()
    for a, b in zip(oh, od):
        assert b.is_cuda
        np.testing.assert_array_equal(a, b.cpu().numpy())


def test_admission_counts_the_library_workspace(ct):
    """A DD backprojection's admission size includes its FP32 scaled
    sinogram: a budget that holds the buffers but not the workspace rejects it."""
    from paper_2503_16741_gb300.serve import Request, Server, request_bytes
    sp = W.scaled(W.circ3d_256(), 64, 90)
    req = Request(gdict(sp), "back", np.zeros(sp.sino_shape, np.float32), projector="dd")
    srv = Server(device=0, slots=2, hbm_budget=request_bytes(req) + (1 << 20))
    assert srv.ex.request_bytes(req) == request_bytes(req) + 4 * int(np.prod(sp.sino_shape))
    with pytest.raises(MemoryError):
        srv.submit(req).result(timeout=30)
    srv.close()
