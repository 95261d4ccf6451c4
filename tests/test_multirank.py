"""The multi-rank host logic of bench.py on CPU: two gloo ranks (one process
each, as torch.distributed.run starts them) agree on the slowest rank's time,
compute the same whole-job value, and own disjoint, contiguous ranges of the
batch's graphs (no data-path collective: each rank refines its own graphs)."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        assert bench._dist() == (ws, rank, rank)
        t = bench.allreduce_max(1.5 + rank, ws, device="cpu")
        start, count = bench.rank_graph_range(rank, 4096)
        ranges = [None] * ws
        dist.all_gather_object(ranges, (start, count))
        q.put((rank, t, ranges, bench.job_value(100.0, ws, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, ranges, value in out:
        assert t == 2.5                               # max over ranks 1.5, 2.5
        assert value == pytest.approx(2 * 100.0 / 2.5)
        assert ranges == [(0, 4096), (4096, 4096)]    # disjoint, contiguous
