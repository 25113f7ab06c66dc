#!/usr/bin/env python
"""Throughput of the separable-footprint (SF-TR) cone-beam projector pair.

One step = SF forward projection y = A x followed by SF backprojection
A^T y over the 3D circular cone-beam workload: 256^3 volume of 0.5 mm voxels,
360 views over 360 deg, flat 512 x 384 detector of 0.8 mm, SAD 785 / SDD 1085
mm, seeded random-ellipsoid phantom (values 0-0.03 / mm).  Metric: giga voxel
updates per second, an update being one (voxel, view) pair, two per pair per
step (forward and back).  Per-step working set (67 MB volume + 283 MB
sinogram) exceeds the 129 MB L2.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 (under torchrun): every rank runs its own replica of the workload
(independent problems, no collective on the data path); value = all ranks'
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SF cone-beam fwd+back GUpdates/s & %HBM roofline; served p50/p99 latency"
UNIT = "GUpdates/s"
WORKLOAD = ("3D circular cone-beam SF-TR forward+back, 256^3 x 0.5 mm FP32 volume, 360 views, "
            "flat 512x384 detector 0.8 mm, SAD 785 / SDD 1085 mm")
# Algorithmic FP32 operations per (voxel, view) update of SF-TR in circular
# geometry, counted from the weight definition (Long et al.'s trapezoid x
# rectangle footprint, amplitude dx |w| / max(|w_x|, |w_y|)):
#   axial centre of the voxel's rectangle (sv k + fv0)          2
#   its row (floor) and the offset of its edges in the row      4
#   the two row bounds (centre -+ half height)                  2
#   the overlaps with the (at most) two rows it meets           6
#   transaxial taps: ~3.8 cells per voxel x one FMA (2)         ~7.6
#   row sums times the axial weights                            2
#   amplitude: wz, w_x^2 + w_y^2 + wz^2, sqrt, x invm, x value  6
#   accumulate into the output                                  2
#                                                       total ~30
# The per-(column, view) trapezoid (~90 operations: four projected corners,
# a sort, the cell integrals) is shared by the column's nz voxels and not
# counted.
SF_FLOPS_PER_UPDATE = 30.0
FP32_LANES = 128  # FP32 FMA lanes per SM (Blackwell)

# Counters of one `ncu --set full` capture of each kernel on this workload
# (per launch): DRAM read + write bytes, L2 (lts__t_sectors x 32) bytes and the
# L2 throughput peak implied by its percent-of-peak counter; src = sha256
# prefix of the kernel's .cu at capture time (the bench reports null once the
# source differs).
NCU = {
    "sf_fwd": {"dram_bytes": 935.3e6, "l2_bytes": 30.472e9, "l2_peak_gbs": 36275.0, "src": "27b5509270244406"},
    "sf_back": {"dram_bytes": 353.1e6, "l2_bytes": 23.183e9, "l2_peak_gbs": 36275.0, "src": "27b5509270244406"},
}


def _src_hash(name: str) -> str:
    p = os.path.join(ROOT, "paper_2503_16741_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [l.split(",") for l in self.lines if l.count(",") >= 8]
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, ws: int, device) -> float:
    """The slowest rank's time (every rank calls it; ws = 1: the time itself)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def job_gupdates(upd_per_step: float, steps: int, ws: int, max_ms: float) -> float:
    """Whole-job throughput: all ranks' updates over the slowest rank's time."""
    return upd_per_step * steps * ws / (max_ms * 1e-3) / 1e9


def cpu_oracle_sample(spec, nviews: int, x=None, threads: int = 0):
    """The FP64 oracle timed on the host cores on a view-decimated copy of
    the workload (nviews evenly spaced views): SF forward + SF back.
    threads = 0: every host core; otherwise that many OpenMP threads."""
    import numpy as np

    import oracle
    import workloads as W
    oracle.build()
    views = np.round(np.arange(nviews) * spec.nview / nviews).astype(int)
    sub = spec.subset(views)
    if x is None:
        x = W.phantom(spec, seed=0)
    every = len(os.sched_getaffinity(0))
    cores = threads or every
    oracle.set_threads(cores)
    try:
        t0 = time.perf_counter()
        y = oracle.forward(sub, "sf", x)
        oracle.back(sub, "sf", y)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(every)
    upd = 2.0 * spec.n_vox * nviews
    return upd / dt / 1e9, dt, cores, f"{nviews} of {spec.nview} views, full volume"


def _gdict(spec):
    return {k: getattr(spec, k) for k in ("kind", "det", "nx", "ny", "nz", "dx", "dy", "dz", "nu",
                                          "nv", "du", "dv", "nview", "theta", "phi", "psi", "sad",
                                          "sdd", "x_src", "z_src", "x_ofst", "y_ofst", "z_ofst",
                                          "u_ofst", "v_ofst")}


SERVE_SIZES = (64, 128, 256, 384, 512)
SERVE_SIZE_P = (0.3, 0.3, 0.2, 0.12, 0.08)
SERVE_VIEWS = (90, 180, 360, 720)


def serving_mix(n_req: int, seed: int = 0):
    """The serving workload: Poisson-arriving requests over the four geometry
    kinds (2D fan beam, circular flat, circular curved, saddle non-circular),
    volumes of 64^3-512^3 (P = 0.3, 0.3, 0.2, 0.12, 0.08; fan beam: (2n)^2
    images; curved: n^2 x n/4, the curved workload's shape), 90 / 180 / 360 /
    720 views, detectors covering the volume (about 2n x 1.5n cells), forward
    40 % / back 40 % / 10-step least-squares MBIR 20 %, SF or DD.  Bounded so
    that 500 requests run in tens of seconds: MBIR volumes at most 256^3
    (non-circular 128^3), non-circular volumes at most 256^3 (the
    non-circular kernels take about ten times longer per update).
    Returns [(request fields, voxel-view updates)]."""
    import numpy as np

    import workloads as W
    rng = np.random.default_rng(seed)
    bases = {"fan2d": W.fan2d_small(720), "circ": W.circ3d_256(720), "curved": W.circ3d_curved(),
             "noncirc": W.noncirc3d_saddle(720)}
    names = list(bases)
    out = []
    for _ in range(n_req):
        name = names[rng.integers(4)]
        n = int(rng.choice(SERVE_SIZES, p=SERVE_SIZE_P))
        views = int(rng.choice(SERVE_VIEWS))
        op = str(rng.choice(["fwd", "back", "mbir"], p=[0.4, 0.4, 0.2]))
        cap = (128 if op == "mbir" else 256) if name == "noncirc" else (256 if op == "mbir" else 512)
        n = min(n, cap)
        spec = W.scaled(bases[name], 2 * n if name == "fan2d" else n, views)
        proj = str(rng.choice(["sf", "dd"]))
        passes = 1 if op != "mbir" else 20
        out.append(({"geometry": _gdict(spec), "op": op, "projector": proj, "iters": 10, "spec": spec},
                    passes * spec.n_vox * spec.nview))
    return out


def serving_bench(dev_index: int, n_req: int, dtype: str, budget: int, loads=(0.9,), n_err: int = 4):
    """Closed-loop saturation, then open-loop Poisson arrivals at the given
    fractions of it, with device-resident inputs and results.  Also the error
    of sampled small results against the FP64 oracle."""
    import numpy as np
    import torch

    import oracle
    from paper_2503_16741_gb300.serve import GpuExecutor, Request, Server, drive, poisson_arrivals
    mix = serving_mix(n_req)
    dev = torch.device("cuda", dev_index)
    T = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[dtype]
    gen = torch.Generator(device=dev).manual_seed(0)
    reqs = []
    for f, _ in mix:
        spec = f["spec"]
        vol = (spec.ny, spec.nx) if spec.kind == "fan2d" else spec.vol_shape
        sino = (spec.nview, spec.nu) if spec.kind == "fan2d" else spec.sino_shape
        shape = vol if f["op"] == "fwd" else sino
        data = torch.rand(shape, generator=gen, device=dev).to(T)  # resident before timing
        reqs.append(Request(f["geometry"], f["op"], data, projector=f["projector"], dtype=dtype,
                            iters=f["iters"], out_device=True))
    ex = GpuExecutor(dev_index, slots=4)
    for r in reqs:  # geometries and MBIR step sizes resident before timing
        ex.geometry(r.geometry)
        if r.op == "mbir":
            ex.step_size(r.geometry, r.projector)
    budget = max(budget, max(ex.request_bytes(r) for r in reqs))  # every request admissible
    srv = Server(hbm_budget=budget, max_batch=4, executor=ex)
    for fut in [srv.submit(r) for r in reqs[:8]]:
        fut.result(timeout=600)
    t0 = time.perf_counter()
    futs = [srv.submit(r) for r in reqs]
    for fut in futs:
        fut.result(timeout=600)
    t_sat = time.perf_counter() - t0
    st_sat = srv.stats()
    srv.close()
    sat_rps = n_req / t_sat
    upd = sum(u for _, u in mix)
    by_load = []
    for load in loads:
        srv = Server(hbm_budget=budget, max_batch=4, executor=ex)
        arr = poisson_arrivals(load * sat_rps, n_req, seed=1)
        t0 = time.perf_counter()
        futs = drive(srv, reqs, arr)
        outs = [fut.result(timeout=600) for fut in futs]
        t_open = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        by_load.append({"load": load, "offered_req_per_s": load * sat_rps, "served_req_per_s": n_req / t_open,
                        "served_gupdates_per_s": upd / t_open / 1e9, "p50_ms": st["p50_ms"],
                        "p99_ms": st["p99_ms"], "launches": st["launches"], "hbm_peak_bytes": st["hbm_peak_bytes"],
                        "memory_waits": st["memory_waits"]})
    # error of sampled small results against FP64 (the oracle on the stored inputs)
    errs = []
    for k, (f, _) in enumerate(mix):
        spec = f["spec"]
        if len(errs) >= n_err or f["op"] not in ("fwd", "back") or spec.n_vox * spec.nview > 3e8:
            continue
        x = reqs[k].data.double().cpu().numpy()
        ref = (oracle.forward if f["op"] == "fwd" else oracle.back)(spec, f["projector"],
                                                                    x.reshape((1,) + x.shape))
        got = outs[k].double().cpu().numpy().reshape(ref.shape)
        errs.append({"request": k, "kind": spec.kind, "det": spec.det, "op": f["op"], "projector": f["projector"],
                     "n": spec.nx, "views": spec.nview,
                     "rel_l2_vs_fp64": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))})
    main = by_load[-1]
    return {"dtype": dtype, "requests": n_req, "hbm_budget_bytes": budget,
            "saturation_req_per_s": sat_rps, "saturation_gupdates_per_s": upd / t_sat / 1e9,
            "saturation_memory_waits": st_sat["memory_waits"], "saturation_hbm_peak_bytes": st_sat["hbm_peak_bytes"],
            "offered_req_per_s": main["offered_req_per_s"], "served_req_per_s": main["served_req_per_s"],
            "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"], "by_load": by_load,
            "error_vs_fp64": errs, "max_rel_l2_vs_fp64": max((e["rel_l2_vs_fp64"] for e in errs), default=None)}


def serving_budget_bound(dev_index: int, n_req: int = 200, budget: int = 512 << 20):
    """FP32 against FP16 storage under an admission budget that binds: the
    same requests (those of the serving mix whose FP32 size fits the budget),
    device-resident, closed loop; served requests per second, the times a
    ready request waited for memory, and the peak admitted bytes."""
    import torch

    from paper_2503_16741_gb300.serve import GpuExecutor, Request, Server
    dev = torch.device("cuda", dev_index)
    ex = GpuExecutor(dev_index, slots=4)
    picked = []
    for f, u in serving_mix(8 * n_req, seed=3):
        probe = Request(f["geometry"], f["op"], None, projector=f["projector"], dtype="f32", iters=f["iters"])
        if ex.request_bytes(probe) <= budget:
            picked.append((f, u))
        if len(picked) == n_req:
            break
    for f, _ in picked:
        if f["op"] == "mbir":
            ex.step_size(f["geometry"], f["projector"])
    out = {"hbm_budget_bytes": budget, "requests": len(picked)}
    for dtype, T in (("f32", torch.float32), ("f16", torch.float16)):
        gen = torch.Generator(device=dev).manual_seed(1)
        reqs = []
        for f, _ in picked:
            spec = f["spec"]
            vol = (spec.ny, spec.nx) if spec.kind == "fan2d" else spec.vol_shape
            sino = (spec.nview, spec.nu) if spec.kind == "fan2d" else spec.sino_shape
            data = torch.rand(vol if f["op"] == "fwd" else sino, generator=gen, device=dev).to(T)
            reqs.append(Request(f["geometry"], f["op"], data, projector=f["projector"], dtype=dtype,
                                iters=f["iters"], out_device=True))
        srv = Server(hbm_budget=budget, max_batch=4, executor=ex)
        for fut in [srv.submit(r) for r in reqs[:8]]:
            fut.result(timeout=600)
        srv.close()
        srv = Server(hbm_budget=budget, max_batch=4, executor=ex)
        t0 = time.perf_counter()
        futs = [srv.submit(r) for r in reqs]
        for fut in futs:
            fut.result(timeout=600)
        dt = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        out[dtype] = {"served_req_per_s": len(reqs) / dt, "served_gupdates_per_s": sum(u for _, u in picked) / dt / 1e9,
                      "memory_waits": st["memory_waits"], "hbm_peak_bytes": st["hbm_peak_bytes"],
                      "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"]}
        del reqs, futs
    out["f16_over_f32"] = out["f16"]["served_req_per_s"] / out["f32"]["served_req_per_s"]
    return out


def run_suite(args):
    """Forward and back time of every projector on each workload (one JSON
    line per case): GUpdates/s per direction at the storage types given."""
    import torch

    import paper_2503_16741_gb300 as ct
    import workloads as W
    from paper_2503_16741_gb300 import build as cbuild
    cbuild.build()
    torch.cuda.set_device(0)
    dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
    cases = [("fan2d 128^2, 180 views, 256 bins", W.fan2d_small(), ["ray", "voxel", "dd", "sf"], ["f32"]),
             ("circ 256^3, 360 views, 512x384", W.circ3d_256(), ["sf", "dd", "voxel", "ray", "sftt"], ["f32", "f16"]),
             ("circ curved 512^2x128, 984 views, 888x64", W.circ3d_curved(), ["dd", "sf"], ["f32"]),
             ("saddle 512^3, 500 views, 1024^2", W.noncirc3d_saddle(), ["sf", "dd", "sftt"], ["f32", "f16", "bf16"])]
    if not args.suite_filter or args.suite_filter in "sinusoidal":
        tv_adam_timing(ct)
    for name, spec, projs, dtypes in cases:
        if args.suite_filter and args.suite_filter not in name:
            continue
        if args.suite_n:  # a smaller copy of the same field of view (profiling captures)
            spec = W.scaled(spec, args.suite_n, args.suite_views or spec.nview)
            name += f" scaled to {spec.nx}x{spec.ny}x{spec.nz}, {spec.nview} views, {spec.nu}x{spec.nv}"
        if args.suite_proj:
            projs = [p for p in projs if p == args.suite_proj]
        if args.suite_dtype:
            dtypes = [t for t in dtypes if t == args.suite_dtype]
        g = ct.Geometry.from_spec(spec)
        for tname in dtypes:
            x = W.phantom(spec, seed=0, device="cuda", dtype=dt[tname])
            x = x.reshape(g.vol_shape)
            y = torch.empty(g.sino_shape, dtype=dt[tname], device="cuda")
            xb = torch.empty(g.vol_shape, dtype=dt[tname], device="cuda")
            for proj in projs:
                ct.forward_into(g, x, y, proj)
                ct.back_into(g, y, xb, proj)
                torch.cuda.synchronize()
                reps = args.suite_reps
                e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                e[0].record()
                for _ in range(reps):
                    ct.forward_into(g, x, y, proj)
                e[1].record()
                for _ in range(reps):
                    ct.back_into(g, y, xb, proj)
                e[2].record()
                torch.cuda.synchronize()
                tf, tb = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
                upd = spec.n_vox * spec.nview
                print(json.dumps({"suite": name, "projector": proj, "dtype": tname,
                                  "fwd_ms": tf, "back_ms": tb, "fwd_gups": upd / tf / 1e6,
                                  "back_gups": upd / tb / 1e6,
                                  "pair_gups": 2 * upd / (tf + tb) / 1e6}), flush=True)
        if spec.kind != "noncirc3d" and (not args.suite_proj or args.suite_proj == "fbp"):
            fbp_timing(ct, g, spec, name, args.suite_reps)
        if "curved" in name and not args.suite_proj:
            mbir_loop_timing(ct, g, spec)
        g.close()


def tv_adam_timing(ct, iters: int = 200):
    """TV-regularised MBIR by Adam through autograd (the objective of Sec. 3)
    on a 200-view sinusoidal trajectory (source z = 20 mm sin 2 theta),
    128^3 volume of 1.6 mm voxels, flat 256 x 192 detector of 1.6 mm, SF."""
    import numpy as np
    import torch
    from paper_2503_16741_gb300.mbir import tv_mbir_adam
    import workloads as W
    nview = 200
    theta = np.linspace(0, 2 * np.pi, nview, endpoint=False)
    spec = W.GeometrySpec("noncirc3d", "flat", 128, 128, 128, 1.6, 1.6, 1.6, 256, 192, 1.6, 1.6, nview,
                          theta=theta, sad=785.0, sdd=1200.0, z_src=20.0 * np.sin(2 * theta))
    g = ct.Geometry.from_spec(spec)
    x_true = W.phantom(spec, seed=0, device="cuda", dtype=torch.float32).reshape(g.vol_shape)
    y = ct.forward(g, x_true, "sf")
    tv_mbir_adam(g, y, "sf", 3, 0.5, 5e-4)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    x, hist = tv_mbir_adam(g, y, "sf", iters, 0.5, 5e-4)
    e[1].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1])
    err = float((x - x_true).double().norm() / x_true.double().norm())
    print(json.dumps({"suite": f"TV-Adam MBIR, {iters} iterations, sinusoidal trajectory 128^3 / 200 views",
                      "ms": ms, "ms_per_iteration": ms / iters, "objective_first_last": [hist[0], hist[-1]],
                      "rel_error": err}), flush=True)
    g.close()


def fbp_timing(ct, g, spec, name: str, reps: int):
    """Filtered backprojection (recon mode): ramp filter and depth-weighted
    voxel-driven backprojection, timed apart, FP32."""
    import torch
    import workloads as W
    x = W.phantom(spec, seed=0, device="cuda", dtype=torch.float32).reshape(g.vol_shape)
    y = ct.forward(g, x, "sf")
    q = torch.empty_like(y)
    xb = torch.empty(g.vol_shape, device="cuda")
    ct.ramp_filter(g, y, out=q)
    ct.back_into(g, q, xb, "voxel", mode="recon")
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    e[0].record()
    for _ in range(reps):
        ct.ramp_filter(g, y, out=q)
    e[1].record()
    for _ in range(reps):
        ct.back_into(g, q, xb, "voxel", mode="recon")
    e[2].record()
    torch.cuda.synchronize()
    tf, tb = e[0].elapsed_time(e[1]) / reps, e[1].elapsed_time(e[2]) / reps
    err = float((xb - x).double().norm() / x.double().norm())
    print(json.dumps({"suite": name, "projector": "fbp (ramp filter + recon back)", "dtype": "f32",
                      "filter_ms": tf, "back_ms": tb, "fbp_ms": tf + tb,
                      "back_gups": spec.n_vox * spec.nview / tb / 1e6,
                      "rel_error_vs_phantom": err}), flush=True)


def mbir_loop_timing(ct, g, spec, steps: int = 10):
    """The 10-step least-squares loop of the curved workload with DD: the
    fused form (two accumulating launches per step) and the same steps taken
    with torch.autograd through the Projector module."""
    import torch
    from paper_2503_16741_gb300.mbir import ls_gradient_descent, ls_step_size
    import workloads as W
    x_true = W.phantom(spec, seed=0, device="cuda", dtype=torch.float32).reshape(g.vol_shape)
    y = ct.forward(g, x_true, "dd")
    lr = ls_step_size(g, "dd")
    A = ct.Projector(g, "proj", "DD", "forward")

    def autograd_loop():
        x = torch.zeros(g.vol_shape, device="cuda", requires_grad=True)
        for _ in range(steps):
            loss = 0.5 * ((A(x) - y) ** 2).sum()
            (gr,) = torch.autograd.grad(loss, [x])
            x.data -= lr * gr
        return x.detach()

    out = {}
    for label, fn in (("fused", lambda: ls_gradient_descent(g, y, "dd", steps, lr=lr)),
                      ("autograd", autograd_loop)):
        fn()
        torch.cuda.synchronize()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        x = fn()
        e[1].record()
        torch.cuda.synchronize()
        ms = e[0].elapsed_time(e[1])
        res = float(((ct.forward(g, x, "dd") - y).double() ** 2).sum() / (y.double() ** 2).sum())
        out[label] = {"ms": ms, "ms_per_step": ms / steps, "rel_residual": res}
    # ordered subsets: 12 interleaved subsets of 82 views, `steps` epochs
    # (an epoch projects every view once each way, like one full step)
    from paper_2503_16741_gb300.mbir import ordered_subsets, os_gradient_descent
    subsets = ordered_subsets(spec.nview, 12)
    lrs = [ls_step_size(g.subset(v), "dd") for v in subsets]
    os_gradient_descent(g, y, "dd", 12, 1, lr=lrs)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    e[0].record()
    x = os_gradient_descent(g, y, "dd", 12, steps, lr=lrs)
    e[1].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1])
    res = float(((ct.forward(g, x, "dd") - y).double() ** 2).sum() / (y.double() ** 2).sum())
    out["ordered_subsets_12"] = {"ms": ms, "ms_per_epoch": ms / steps, "rel_residual": res}
    upd = 2 * steps * spec.n_vox * spec.nview
    print(json.dumps({"suite": "10-step least-squares loop, DD, curved 512^2x128 / 984 views",
                      "fused": out["fused"], "autograd": out["autograd"],
                      "ordered_subsets_12": out["ordered_subsets_12"],
                      "fused_gups": upd / out["fused"]["ms"] / 1e6}), flush=True)


def saddle_record(dev, reps: int = 2):
    """The non-circular saddle workload (512^3 volume of 0.4 mm voxels, 500
    views, flat 1024^2 detector of 0.4 mm; saddle trajectory with seeded pose
    jitter) with SF-TR: forward and back time (CUDA events, after one warm-up
    pair) in FP32 and in FP16 storage, and the FP16 results' error against
    the FP64 oracle: the forward on two views (input and output rounding
    included) and the back at 200 sampled voxels of the stored sinogram."""
    import numpy as np
    import torch

    import oracle
    import paper_2503_16741_gb300 as ct
    import workloads as W
    spec = W.noncirc3d_saddle()
    g = ct.Geometry.from_spec(spec)
    x64 = W.phantom(spec, seed=0, device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    upd = spec.n_vox * spec.nview
    rec = {"workload": "non-circular saddle cone beam, 512^3 x 0.4 mm, 500 views, flat 1024^2 x 0.4 mm, "
                       "SAD 785 / SDD 1200 mm, SF-TR", "updates_per_op": upd}
    for name, dt in (("f32", torch.float32), ("f16", torch.float16)):
        x = x64.to(dt).reshape(g.vol_shape)
        y = torch.empty(g.sino_shape, dtype=dt, device=dev)
        xb = torch.empty(g.vol_shape, dtype=dt, device=dev)
        ct.forward_into(g, x, y, "sf", stream=stream)
        ct.back_into(g, y, xb, "sf", stream=stream)
        torch.cuda.synchronize(dev)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        tf = tb = 0.0
        for _ in range(reps):
            e[0].record(stream)
            ct.forward_into(g, x, y, "sf", stream=stream)
            e[1].record(stream)
            ct.back_into(g, y, xb, "sf", stream=stream)
            e[2].record(stream)
            torch.cuda.synchronize(dev)
            tf += e[0].elapsed_time(e[1]) / reps
            tb += e[1].elapsed_time(e[2]) / reps
        r = {"fwd_ms": tf, "back_ms": tb, "fwd_gups": upd / tf / 1e6, "back_gups": upd / tb / 1e6,
             "pair_gups": 2 * upd / (tf + tb) / 1e6}
        if name == "f16":
            views = [123, 377]
            xn = x64.cpu().numpy()
            yref = oracle.forward(spec.subset(views), "sf", xn)
            yv = y[views].double().cpu().numpy()
            r["fwd_rel_l2_vs_fp64"] = float(np.linalg.norm(yv - yref) / np.linalg.norm(yref))
            sel = np.random.default_rng(3).choice(spec.n_vox, size=200, replace=False)
            bref = oracle.back_voxels(spec, "sf", y.double().cpu().numpy(), sel)
            bgot = xb.double().cpu().numpy().ravel()[sel]
            r["back_rel_l2_vs_fp64"] = float(np.linalg.norm(bgot - bref) / np.linalg.norm(bref))
            r["error_sample"] = "forward: views 123, 377 of the FP64 phantom; back: 200 voxels of the stored sinogram"
        rec[name] = r
        del x, y, xb
    g.close()
    return rec


def run_reference(args):
    """The oracle as the reference arm: K timed steps of a bounded sample."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import workloads as W
    spec = W.circ3d_256()
    x = W.phantom(spec, seed=0)
    nviews = args.ref_views
    for _ in range(args.warmup):
        cpu_oracle_sample(spec, nviews, x)
    t = 0.0
    for _ in range(args.steps):
        _, dt, cores, sample = cpu_oracle_sample(spec, nviews, x)
        t += dt
    upd = 2.0 * spec.n_vox * nviews * args.steps
    val = upd / t / 1e9
    out = {"metric": METRIC, "value": val, "unit": UNIT, "impl": "reference", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD + f" (oracle sample: {sample})"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-views", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=500)
    ap.add_argument("--serve-budget-gib", type=float, default=5.0,
                    help="admission budget, GiB (5: just above the largest FP32 request of the mix)")
    ap.add_argument("--serve-loads", default="0.9", help="open-loop loads, fractions of saturation (comma list)")
    ap.add_argument("--no-saddle", action="store_true", help="skip the non-circular saddle record")
    ap.add_argument("--saddle-reps", type=int, default=2)
    ap.add_argument("--suite", action="store_true", help="time every projector on each workload")
    ap.add_argument("--suite-reps", type=int, default=2)
    ap.add_argument("--suite-filter", default="", help="only workloads whose name contains this")
    ap.add_argument("--suite-n", type=int, default=0, help="scale each suite workload to n voxels per side")
    ap.add_argument("--suite-views", type=int, default=0, help="view count of a scaled suite workload")
    ap.add_argument("--suite-proj", default="", help="only this projector")
    ap.add_argument("--suite-dtype", default="", help="only this storage type")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.suite:
        return run_suite(args)

    import torch
    import torch.distributed as dist

    import paper_2503_16741_gb300 as ct
    import workloads as W
    from paper_2503_16741_gb300 import build as cbuild

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cbuild.build()
    dev = torch.device("cuda", local)
    spec = W.circ3d_256()
    geom = ct.Geometry.from_spec(spec)
    x = W.phantom(spec, seed=0, device=dev, dtype=torch.float32)
    y = torch.empty(spec.sino_shape, dtype=torch.float32, device=dev)
    xb = torch.empty(spec.vol_shape, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        ct.forward_into(geom, x, y, "sf", stream=stream)
        ct.back_into(geom, y, xb, "sf", stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for k in range(K):
        ev[k][0].record(stream)
        ct.forward_into(geom, x, y, "sf", stream=stream)
        ev[k][1].record(stream)
        ct.back_into(geom, y, xb, "sf", stream=stream)
        ev[k][2].record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    fwd_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / K
    back_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / K
    total_ms = max_over_ranks(ev[0][0].elapsed_time(ev[-1][2]), ws, dev)
    upd_step = 2.0 * spec.n_vox * spec.nview
    value = job_gupdates(upd_step, K, ws, total_ms)

    # end to end through the public API with host buffers (pinned), timed by
    # the host's wall clock: each step copies the volume in, projects forward
    # and back, copies the result volume out and waits for it on the host
    xh = x.cpu().pin_memory()
    xbh = torch.empty(spec.vol_shape, dtype=torch.float32).pin_memory()
    xd = torch.empty_like(x)

    def e2e_step():
        xd.copy_(xh, non_blocking=True)
        ct.forward_into(geom, xd, y, "sf", stream=stream)
        ct.back_into(geom, y, xb, "sf", stream=stream)
        xbh.copy_(xb, non_blocking=True)
        torch.cuda.synchronize(dev)

    for _ in range(2):
        e2e_step()
    if ws > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_step()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, ws, dev)
    e2e = {"value": job_gupdates(upd_step, K, ws, e2e_ms), "unit": UNIT,
           "h2d_bytes_per_step": xh.numel() * 4, "d2h_bytes_per_step": xbh.numel() * 4,
           "timer": "host wall clock, synchronised every step"}

    if rank != 0:
        return
    peaks = _peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = n_sm * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s at the sampled clock
    dom, dom_ms, dom_src = ("sf_back", back_ms, "k_sf.cu") if back_ms >= fwd_ms else \
        ("sf_fwd", fwd_ms, "k_sf.cu")
    flops = SF_FLOPS_PER_UPDATE * spec.n_vox * spec.nview
    achieved = flops / (dom_ms * 1e-3) / 1e12
    nc = NCU.get(dom)
    fresh = nc is not None and nc.get("src") == _src_hash(dom_src)
    traffic = nc["dram_bytes"] if fresh else None
    vol_b, sino_b = spec.n_vox * 4, spec.n_cells * 4
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_ach = (vol_b + sino_b) / (dom_ms * 1e-3) / 1e9
    mem = {"dram_bytes": traffic, "dram_gbs": None, "dram_frac": None, "l2_bytes": None,
           "l2_gbs": None, "l2_peak_gbs": None, "l2_frac": None,
           "note": "ncu counters of the same kernel source, per launch, over this run's kernel time; "
                   "DRAM against the measured copy bandwidth, L2 against the peak implied by ncu's "
                   "lts__t_sectors percent of peak" if fresh else "no capture of the current source"}
    if fresh:
        mem["dram_gbs"] = traffic / (dom_ms * 1e-3) / 1e9
        mem["dram_frac"] = mem["dram_gbs"] / hbm_peak
        mem["l2_bytes"] = nc["l2_bytes"]
        mem["l2_gbs"] = nc["l2_bytes"] / (dom_ms * 1e-3) / 1e9
        mem["l2_peak_gbs"] = nc["l2_peak_gbs"]
        mem["l2_frac"] = mem["l2_gbs"] / nc["l2_peak_gbs"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": max(args.warmup, 3), "ms_per_step": total_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "projector": "SF-TR", "batch": 1,
                   "l2": "inputs larger than L2 (67 MB volume + 283 MB sinogram per step)",
                   "fwd_ms": fwd_ms, "back_ms": back_ms},
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved,
                     "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                     "traffic": traffic, "memory": mem,
                     "peak_note": f"FP32 FMA peak {n_sm} SM x {FP32_LANES} lanes x 2 at {sm_mhz:.0f} MHz",
                     "flops_per_update": SF_FLOPS_PER_UPDATE},
        "hbm_roofline": {"kernel": dom, "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s",
                         "frac": hbm_ach / hbm_peak, "bytes": "compulsory: read input once, write output once",
                         "peak_note": "of measured (MEASURED_PEAKS.json hbm_gbs)"},
        "e2e": e2e,
        "gpu_launches": 3 * K,  # per step: z-major copy, SF forward, SF back
        "clocks": clk,
    }
    if not args.no_serving:
        torch.cuda.synchronize(dev)
        budget = int(args.serve_budget_gib * (1 << 30))
        loads = tuple(float(v) for v in args.serve_loads.split(","))
        out["serving"] = [serving_bench(local, args.serve_requests, "f32", budget, loads),
                          serving_bench(local, args.serve_requests, "f16", budget, loads)]
        out["serving_budget_bound"] = serving_budget_bound(local)
        out["serving_mix"] = (serving_mix.__doc__.split("Returns")[0].strip().replace("\n    ", " ")
                              + " Inputs and results device-resident; open-loop Poisson arrivals at "
                              f"{args.serve_loads} of the measured closed-loop saturation (top-level figures at "
                              f"the last); the same {args.serve_budget_gib:g} GiB admission budget (request "
                              "buffers, temporaries and library workspace) for both storage types.")
    if not args.no_saddle:
        out["saddle"] = saddle_record(dev, args.saddle_reps)
    if ws == 1 and not args.no_cpu_baseline:
        val, dt, cores, sample = cpu_oracle_sample(spec, 8)
        val1, dt1, _, sample1 = cpu_oracle_sample(spec, 2, threads=1)
        out["cpu_baseline"] = {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample + f" ({dt:.1f} s)",
                               "one_core": {"value": val1, "unit": UNIT, "cores": 1,
                                            "sample": sample1 + f" ({dt1:.1f} s)"}}
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
