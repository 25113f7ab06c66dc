"""The multi-rank path of bench.py (every rank a replica, the slowest rank's
time, whole-job throughput) on CPU with the gloo backend, world size 2."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, local = bench._dist()
        ms = bench.max_over_ranks(10.0 * (rank + 1), w, "cpu")
        out[rank] = (w, r, local, ms, bench.job_gupdates(1e9, 4, w, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        w, r, local, ms, val = res[rank]
        assert (w, r, local) == (ws, rank, rank)
        assert ms == 20.0  # the slower rank's 20 ms, on both ranks
        assert val == pytest.approx(1e9 * 4 * ws / 20e-3 / 1e9)


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_gupdates(2e9, 10, 1, 100.0) == pytest.approx(200.0)
