"""The multi-GPU form of bench.py is independent replicas: only a barrier and a
max of the per-rank times cross ranks (each rank evaluates its own walkers
over the whole catalog, so no data-path collective is built).
This checks those cross-rank pieces with two gloo ranks on the CPU: the
environment is read as torchrun sets it, the barrier holds every rank, and
the time each rank reports is the slowest rank's (the job's time), so that
value = units of all ranks / that time.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import time

    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    t0 = time.perf_counter()
    if r == 1:
        time.sleep(0.3)  # the slow rank
    bench.barrier(w)
    waited = time.perf_counter() - t0
    mine = 1.0 + r  # per-rank timed seconds
    q.put((r, w, local, waited, bench.allmax(w, mine)))
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert [o[2] for o in out] == [0, 1]
    assert out[0][3] >= 0.25  # rank 0 waited for the slow rank at the barrier
    assert all(o[4] == pytest.approx(2.0) for o in out)  # every rank holds the max


def test_single_rank_is_the_identity(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup() == (1, 0, 0)
    bench.barrier(1)
    assert bench.allmax(1, 3.5) == 3.5
