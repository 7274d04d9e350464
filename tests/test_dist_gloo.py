"""The multi-process benchmark path on CPU: world size 2 over gloo.

ES does not shard across GPUs here (every run has one GPU), so bench.py
--gpus N runs N independent replicas with a barrier on both sides of the
timed region and the maximum time over ranks; this checks that plumbing
(rendezvous on 127.0.0.1, barrier, max over ranks, rank-0-only reference
arm) with two CPU processes.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    ws, r, local = bench.dist_setup(2)
    assert ws == 2 and r == rank and dist.get_backend() == "gloo"
    bench.barrier(ws)
    mx = bench.max_over_ranks(10.0 * (rank + 1), ws)
    bench.barrier(ws)
    dist.destroy_process_group()
    q.put((rank, mx))


def test_two_rank_barrier_and_max():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 20.0), (1, 20.0)]
