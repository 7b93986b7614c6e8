"""The multi-rank bench logic on CPU (gloo, world size 2): each rank runs its
own replica, the whole-job value is the pairs of all ranks over the slowest
rank's time, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [1500.0, 2500.0][rank]
        pairs = [200, 200][rank]
        t_max, pairs_all = bench.aggregate_ranks(ms, pairs, world)

        class Args:
            n = 0
            warmup = 0
            steps = 1

        ref = bench.run_reference(Args(), rank, world) if rank == 1 else "skipped"
        q.put((rank, t_max, pairs_all, ref))
    finally:
        dist.destroy_process_group()


def test_aggregate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, pairs_all, ref in out:
        assert t_max == 2500.0            # slowest rank's time
        assert pairs_all == 400.0         # all ranks' pairs
    assert out[1][3] is None              # the reference arm: rank 0 only, others return no line


def test_aggregate_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(123.0, 7, 1) == (123.0, 7.0)
