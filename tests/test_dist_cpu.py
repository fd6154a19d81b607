"""bench.py's multi-process plumbing on CPU: two gloo ranks (world size 2).

The batched path shards as independent replicas (each rank solves its own
batches, no collective on the data path); bench.py only needs a barrier and
max / sum reductions of its timings and counts, checked here.
"""
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


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    t = bench.max_over_ranks(w, 1.0 + r)          # slowest rank's time
    solves = bench.sum_over_ranks(w, 1024 * (r + 1))
    q.put((r, w, local, t, solves, solves / t))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_bench():
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
    for r, (rank, world, local, t, solves, value) in enumerate(out):
        assert (rank, world, local) == (r, 2, r)
        assert t == 2.0 and solves == 3072.0 and value == pytest.approx(1536.0)


def test_single_process_defaults():
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        os.environ.pop(k, None)
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(1, 3.5) == 3.5 and bench.sum_over_ranks(1, 7) == 7
