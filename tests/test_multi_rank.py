"""The multi-rank (replica) path of bench.py on CPU: two gloo ranks.

bench.py runs one independent replica per GPU; ranks meet only at barriers
and in one max-reduction of their timed region.  This test runs that host
logic with world size 2 on the gloo backend (no GPU)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, ws: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        bench._barrier(ws)
        ms = 2.0 + 3.0 * rank                       # rank 1 is the slow one
        ms_max = bench._barrier_max(ms, ws)
        value = bench.whole_job_value(1_000_000, ws, ms_max)
        q.put((rank, got_ws, got_rank, got_local, ms_max, value))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=5) for _ in range(ws))
    for rank, got_ws, got_rank, got_local, ms_max, value in res:
        assert (got_ws, got_rank, got_local) == (ws, rank, rank)
        assert ms_max == 5.0                        # max over ranks
        assert value == pytest.approx(2 * 1_000_000 / 5e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._barrier_max(3.5, 1) == 3.5
    assert bench.whole_job_value(10, 1, 2.0) == pytest.approx(5000.0)
