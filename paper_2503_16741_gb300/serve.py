"""Continuous-batching projection server.

Requests -- a forward projection, a backprojection or a short MBIR solve
(least-squares gradient descent, Sec. 2.4) on any geometry of Sec. 2.2 --
arrive at any time from any thread.  A scheduler thread admits them while a
slot (a CUDA stream) is free and the device memory they need fits the HBM
budget, so requests that arrive while others run start as soon as resources
free up and their work overlaps on the device.  Waiting requests with the
same geometry, operation, projector and storage type are merged into one
batched launch (the kernels treat batch items independently and
deterministically, so each result is the same alone and in a batch).
Geometry tables stay resident on the device between requests, and a request
may carry a device tensor and ask for its result on the device, so volumes
and sinograms stay resident too.  Admission counts every byte a request
holds on the device while it runs: its input, output and temporaries and the
library's pooled workspace (ct_workspace_bytes), whose pool is capped at the
budget.

The scheduler is independent of the device: `Scheduler` drives an
`Executor` (launch a group, poll it, collect results).  `GpuExecutor` runs
the library's kernels; tests drive the scheduler with a host-only executor.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Any, Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

OPS = ("fwd", "back", "mbir", "fbp")
ITEMSIZE = {"f32": 4, "f16": 2, "bf16": 2}


@dataclasses.dataclass(eq=False)
class Request:
    """One job.  `geometry`: keyword arguments of `Geometry` (hashable once
    frozen by `geometry_key`).  `data`: the volume (fwd) or the sinogram
    (back, mbir, fbp), shape (nz, ny, nx) / (nview, nv, nu) (2D: without the
    z / v axis), as a host array or as a tensor already on the server's
    device (used in place: no host copy).  `dtype`: storage type on the
    device.  `out_device`: return the result as a device tensor instead of a
    host array.  `fbp` reconstructs by filtered backprojection (the projector
    is the recon mode's voxel-driven one whatever `projector` says)."""
    geometry: Dict[str, Any]
    op: str
    data: Any
    projector: str = "sf"
    dtype: str = "f32"
    iters: int = 10
    deadline_s: Optional[float] = None
    out_device: bool = False


def geometry_key(geom: Dict[str, Any]) -> Tuple:
    items = []
    for k in sorted(geom):
        v = geom[k]
        if isinstance(v, np.ndarray) or isinstance(v, (list, tuple)):
            v = tuple(np.asarray(v, dtype=np.float64).ravel().tolist())
        items.append((k, v))
    return tuple(items)


def shapes(geom: Dict[str, Any]):
    two_d = geom["kind"] == "fan2d"
    vol = (geom["ny"], geom["nx"]) if two_d else (geom["nz"], geom["ny"], geom["nx"])
    sino = (geom["nview"], geom["nu"]) if two_d else (geom["nview"], geom["nv"], geom["nu"])
    return vol, sino


def _on_device(data) -> bool:
    return getattr(data, "is_cuda", False)


def request_bytes(req: Request) -> int:
    """Device bytes of a request's own buffers while it runs: input, output
    and, for MBIR and FBP, the FP32 residual or filtered sinogram.  (The
    GPU executor adds the library's pooled workspace.)"""
    vol, sino = shapes(req.geometry)
    nv, ns = int(np.prod(vol)), int(np.prod(sino))
    it = ITEMSIZE[req.dtype]
    if req.op == "fwd":
        return (nv + ns) * it
    if req.op == "back":
        return (ns + nv) * it
    if req.op == "fbp":
        return (ns + nv) * it + ns * 4
    return (ns + nv) * it + ns * 4


def group_key(req: Request) -> Tuple:
    return (geometry_key(req.geometry), req.op, req.projector, req.dtype,
            req.iters if req.op == "mbir" else 0, _on_device(req.data), req.out_device)


@dataclasses.dataclass(eq=False)
class _Pending:
    req: Request
    fut: cf.Future
    t_submit: float
    nbytes: int


class Executor:
    """Runs groups of compatible requests.  launch() returns a handle;
    done(handle) polls it; results(handle) returns one host array per
    request; release(handle) frees its device memory."""

    slots = 1

    def request_bytes(self, req: Request) -> int:
        """Device bytes the request holds while it runs (admission)."""
        return request_bytes(req)

    def launch(self, slot: int, reqs: Sequence[Request]):  # pragma: no cover - interface
        raise NotImplementedError

    def done(self, handle) -> bool:  # pragma: no cover - interface
        raise NotImplementedError

    def results(self, handle) -> List[np.ndarray]:  # pragma: no cover - interface
        raise NotImplementedError

    def release(self, handle) -> None:
        pass


class Scheduler:
    """Admission (slots, HBM budget, FIFO with grouping), completion
    polling, deadlines and cancellation."""

    def __init__(self, executor: Executor, hbm_budget: int, max_batch: int = 8,
                 group_window: int = 64, poll_s: float = 2e-4):
        self.ex = executor
        self.budget = int(hbm_budget)
        self.max_batch = max_batch
        self.group_window = group_window
        self.poll_s = poll_s
        self._lock = threading.Condition()
        self._queue: collections.deque = collections.deque()
        self._free_slots = list(range(executor.slots))
        self._inflight: List[Tuple[Any, int, List[_Pending], int]] = []
        self.in_use = 0
        self.peak_in_use = 0
        self.latencies: List[float] = []
        self.completed = 0
        self.rejected = 0
        self.timed_out = 0
        self.launches = 0
        self.memory_waits = 0  # admissions deferred because the budget was full while a slot was free
        self._waiting_head = None
        self._stop = False
        self._thread = threading.Thread(target=self._run, name="ct-scheduler", daemon=True)
        self._thread.start()

    # ---- client side
    def submit(self, req: Request) -> cf.Future:
        fut: cf.Future = cf.Future()
        if req.op not in OPS:
            fut.set_exception(ValueError(f"unknown op {req.op!r}"))
            return fut
        try:
            nbytes = self.ex.request_bytes(req)
        except Exception as e:  # noqa: BLE001 - a request the executor cannot size is rejected
            fut.set_exception(e)
            return fut
        with self._lock:
            if nbytes > self.budget:
                self.rejected += 1
                fut.set_exception(MemoryError(
                    f"request needs {nbytes} bytes, above the HBM budget of {self.budget}"))
                return fut
            self._queue.append(_Pending(req, fut, time.perf_counter(), nbytes))
            self._lock.notify()
        return fut

    def queue_depth(self) -> int:
        with self._lock:
            return len(self._queue)

    def close(self, wait: bool = True):
        with self._lock:
            self._stop = True
            self._lock.notify()
        if wait:
            self._thread.join()

    def stats(self) -> Dict[str, Any]:
        with self._lock:
            lat = np.array(self.latencies) if self.latencies else np.zeros(1)
            return {"completed": self.completed, "rejected": self.rejected,
                    "timed_out": self.timed_out, "launches": self.launches,
                    "p50_ms": float(np.percentile(lat, 50) * 1e3),
                    "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "hbm_peak_bytes": self.peak_in_use, "queue_depth": len(self._queue),
                    "memory_waits": self.memory_waits}

    # ---- scheduler thread
    def _take_group(self) -> Optional[List[_Pending]]:
        """Head of the queue plus compatible requests among the next
        group_window waiting ones, within max_batch and the free budget."""
        while self._queue and self._queue[0].fut.cancelled():
            self._queue.popleft()
        if not self._queue:
            return None
        head = self._queue[0]
        if self.in_use + head.nbytes > self.budget:
            if head is not self._waiting_head:  # count each deferred head once
                self._waiting_head = head
                self.memory_waits += 1
            return None
        key = group_key(head.req)
        group, total = [head], head.nbytes
        for p in list(self._queue)[1:self.group_window]:
            if len(group) >= self.max_batch:
                break
            if p.fut.cancelled() or group_key(p.req) != key:
                continue
            if self.in_use + total + p.nbytes > self.budget:
                break
            group.append(p)
            total += p.nbytes
        for p in group:
            self._queue.remove(p)
        return group

    def _complete(self, handle, slot, group, nbytes):
        try:
            outs = self.ex.results(handle)
            err = None
        except Exception as e:  # noqa: BLE001 - reported on every future of the group
            outs, err = None, e
        self.ex.release(handle)
        now = time.perf_counter()
        with self._lock:
            self.in_use -= nbytes
            self._free_slots.append(slot)
            for k, p in enumerate(group):
                if p.fut.done():
                    continue
                if err is not None:
                    p.fut.set_exception(err)
                else:
                    p.fut.set_result(outs[k])
                    self.latencies.append(now - p.t_submit)
                    self.completed += 1

    def _run(self):
        while True:
            progressed = False
            # completions and deadlines
            for item in list(self._inflight):
                handle, slot, group, nbytes = item
                if self.ex.done(handle):
                    self._inflight.remove(item)
                    self._complete(handle, slot, group, nbytes)
                    progressed = True
                else:
                    now = time.perf_counter()
                    for p in group:
                        if (p.req.deadline_s is not None and not p.fut.done()
                                and now - p.t_submit > p.req.deadline_s):
                            p.fut.set_exception(TimeoutError("deadline passed before completion"))
                            with self._lock:
                                self.timed_out += 1
            # admissions (the launch itself runs outside the lock so that
            # clients can keep submitting)
            while True:
                with self._lock:
                    if not self._free_slots:
                        break
                    group = self._take_group()
                    if group is None:
                        break
                    slot = self._free_slots.pop()
                    nbytes = sum(p.nbytes for p in group)
                    self.in_use += nbytes
                    self.peak_in_use = max(self.peak_in_use, self.in_use)
                try:
                    handle = self.ex.launch(slot, [p.req for p in group])
                except Exception as e:  # noqa: BLE001 - a failed launch rejects its group
                    with self._lock:
                        self.in_use -= nbytes
                        self._free_slots.append(slot)
                        self.rejected += len(group)
                    for p in group:
                        if not p.fut.done():
                            p.fut.set_exception(e)
                    continue
                with self._lock:
                    self.launches += 1
                self._inflight.append((handle, slot, group, nbytes))
                progressed = True
            with self._lock:
                if self._stop and not self._queue and not self._inflight:
                    return
                if not progressed:
                    self._lock.wait(timeout=self.poll_s)


class GpuExecutor(Executor):
    """Runs groups on one GPU with the library's kernels: one CUDA stream
    per slot; pinned host staging; geometries cached on the device; MBIR
    steps fused into ct_forward_acc / ct_back_acc."""

    def __init__(self, device: int = 0, slots: int = 4):
        import torch

        from .binding import Geometry
        self.torch = torch
        self.Geometry = Geometry
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.slots = slots
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self._geoms: Dict[Tuple, Any] = {}
        self._lr: Dict[Tuple, float] = {}
        self._dt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
        self._pinned: Dict[Tuple, List[Any]] = collections.defaultdict(list)
        self._plock = threading.Lock()

    def _pinned_buffer(self, shape, dtype):
        """A pinned host buffer from a pool keyed by shape and dtype
        (page-locking memory per request would cost more than the copy)."""
        key = (tuple(shape), dtype)
        with self._plock:
            if self._pinned[key]:
                return self._pinned[key].pop()
        return self.torch.empty(shape, dtype=dtype).pin_memory()

    def _return_pinned(self, buf):
        with self._plock:
            self._pinned[(tuple(buf.shape), buf.dtype)].append(buf)

    def request_bytes(self, req: Request) -> int:
        """The request's buffers plus the library workspace its calls take
        (the larger of the forward's and the back's for MBIR: they run one
        after the other on one stream, whose pool reuses the memory)."""
        from .binding import workspace_bytes
        g = self.geometry(req.geometry)
        dt = self._dt[req.dtype]
        if req.op == "fwd":
            ws = workspace_bytes(g, req.projector, "fwd", dt)
        elif req.op == "back":
            ws = workspace_bytes(g, req.projector, "back", dt)
        elif req.op == "mbir":
            ws = max(workspace_bytes(g, req.projector, "fwd", dt),
                     workspace_bytes(g, req.projector, "back", self.torch.float32))
        else:
            ws = workspace_bytes(g, "voxel", "back", self.torch.float32, mode="recon")
        return request_bytes(req) + ws

    def geometry(self, g: Dict[str, Any]):
        key = geometry_key(g)
        if key not in self._geoms:
            self.torch.cuda.set_device(self.device)
            self._geoms[key] = self.Geometry(**g)
        return self._geoms[key]

    def step_size(self, g: Dict[str, Any], projector: str) -> float:
        from .mbir import ls_step_size
        key = (geometry_key(g), projector)
        if key not in self._lr:
            self._lr[key] = ls_step_size(self.geometry(g), projector)
        return self._lr[key]

    def launch(self, slot: int, reqs: Sequence[Request]):
        from .binding import back_into, forward_into, ramp_filter
        from .mbir import ls_gradient_descent
        torch = self.torch
        torch.cuda.set_device(self.device)
        r0 = reqs[0]
        geom = self.geometry(r0.geometry)
        lr = self.step_size(r0.geometry, r0.projector) if r0.op == "mbir" else None
        vol, sino = shapes(r0.geometry)
        in_shape = vol if r0.op == "fwd" else sino
        for r in reqs:
            if tuple(r.data.shape) != tuple(in_shape):
                raise ValueError(f"input shape {r.data.shape} != {in_shape}")
        dt = self._dt[r0.dtype]
        stream = self.streams[slot]
        resident = _on_device(r0.data)
        host_in = None
        if not resident:
            host_in = self._pinned_buffer((len(reqs),) + tuple(in_shape), dt)
            for k, r in enumerate(reqs):
                host_in[k].copy_(torch.from_numpy(np.asarray(r.data, dtype=np.float32)))
        tmp = None  # a stream-ordered temporary that must outlive the launch
        with torch.cuda.stream(stream):
            if resident:  # device tensors: used in place (stacked when batched)
                stream.wait_stream(torch.cuda.current_stream(self.device))
                d_in = (r0.data.to(dt).reshape((1,) + tuple(in_shape)) if len(reqs) == 1 else
                        torch.stack([r.data.to(dt) for r in reqs]))
            else:
                d_in = host_in.to(self.device, non_blocking=True)
            if r0.op == "fwd":
                d_out = torch.empty((len(reqs),) + sino, dtype=dt, device=self.device)
                forward_into(geom, d_in, d_out, r0.projector, stream=stream)
            elif r0.op == "back":
                d_out = torch.empty((len(reqs),) + vol, dtype=dt, device=self.device)
                back_into(geom, d_in, d_out, r0.projector, stream=stream)
            elif r0.op == "fbp":
                tmp = torch.empty(d_in.shape, dtype=torch.float32, device=self.device)
                ramp_filter(geom, d_in, out=tmp, stream=stream)
                d_out = torch.empty((len(reqs),) + vol, dtype=dt, device=self.device)
                back_into(geom, tmp, d_out, "voxel", mode="recon", stream=stream)
            else:
                d_out = ls_gradient_descent(geom, d_in, r0.projector, r0.iters, lr=lr, stream=stream)
            host_out = None
            if not r0.out_device:
                host_out = self._pinned_buffer(tuple(d_out.shape), dt)
                host_out.copy_(d_out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        # keep device buffers alive until the event has passed
        return {"event": ev, "host_out": host_out, "host_in": host_in, "keep": (d_in, d_out, tmp),
                "device_out": d_out if r0.out_device else None}

    def done(self, handle) -> bool:
        return handle["event"].query()

    def results(self, handle) -> List[Any]:
        if handle.get("device_out") is not None:  # device-resident results (ready: the event passed)
            d = handle["device_out"]
            return [d[k] for k in range(d.shape[0])]
        out = handle["host_out"].float().numpy()
        return [out[k].copy() for k in range(out.shape[0])]

    def release(self, handle) -> None:
        handle["keep"] = None
        handle["device_out"] = None
        for k in ("host_in", "host_out"):
            if handle.get(k) is not None:
                self._return_pinned(handle[k])
                handle[k] = None


class Server(Scheduler):
    """A Scheduler over a GpuExecutor (pass `executor` to keep its resident
    geometries, step sizes and pinned buffers across servers)."""

    def __init__(self, device: int = 0, slots: int = 4, hbm_budget: int = 32 << 30,
                 max_batch: int = 8, executor: Optional[GpuExecutor] = None, **kw):
        ex = executor or GpuExecutor(device, slots)
        # the library's pool keeps no more freed workspace than the budget
        from .binding import workspace_limit
        ex.torch.cuda.set_device(ex.device)
        workspace_limit(hbm_budget)
        super().__init__(ex, hbm_budget, max_batch=max_batch, **kw)


def poisson_arrivals(rate_hz: float, n: int, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, n))


def drive(sched: Scheduler, reqs: Sequence[Request], arrivals: Sequence[float],
          clock: Callable[[], float] = time.perf_counter) -> List[cf.Future]:
    """Submit each request at its arrival time (relative to now)."""
    t0 = clock()
    futs = []
    for r, t in zip(reqs, arrivals):
        while clock() - t0 < t:
            time.sleep(min(1e-3, max(0.0, t - (clock() - t0))))
        futs.append(sched.submit(r))
    return futs
