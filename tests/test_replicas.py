"""bench.py's multi-rank path (replicas, one per GPU): the whole-job rate is the sum of
the units all ranks processed over the slowest rank's time.  Run here as two gloo
ranks on the CPU."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    w, r, _, pg = bench.dist_setup()
    try:
        rate = bench.replica_throughput(units=100.0 * (rank + 1), seconds=0.5 + rank, pg=pg)
        mx = bench.max_over_ranks(float(rank), pg)
        q.put((r, w, rate, mx))
    finally:
        pg.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    pytest.importorskip("torch.distributed")
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
    # units 100 + 200 over the slowest time 1.5 s
    assert [o[:2] for o in out] == [(0, 2), (1, 2)]
    assert all(abs(o[2] - 200.0) < 1e-9 for o in out)
    assert all(o[3] == 1.0 for o in out)


def test_single_process_needs_no_process_group():
    import bench
    assert bench.replica_throughput(300.0, 1.5, None) == 200.0
