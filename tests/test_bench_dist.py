"""bench.py's multi-rank logic on CPU (gloo, world size 2): every rank runs a
replica; the job's time is the slowest rank's and its throughput the sum of
all ranks' queries over that time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    dist = bench.dist_init(w, "gloo")
    t = bench.max_over_ranks(1.0 + rank, dist)          # rank 1 is slower
    q = bench.sum_over_ranks(10_000.0, dist)            # each rank searched its own 10,000 queries
    out.put((r, w, local, t, q, q / t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, local, t, q, v) in enumerate(res):
        assert (r, w, local) == (rank, 2, rank)
        assert t == 2.0 and q == 20_000.0 and v == 10_000.0


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5 and bench.sum_over_ranks(7.0, None) == 7.0
