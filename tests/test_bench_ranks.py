"""The multi-GPU form of the benchmark on CPU: world size 2 over gloo.

Independent replicas shard over ranks (no collective on the data path): each rank
runs its own R replicas with distinct run ids, the step time is the slowest rank's
and the point-steps are summed over ranks.
"""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, runs = bench.runs_of("c2", 3, rank)
        ids = [r["cfg"]["run_id"] for r in runs]
        t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
        n = bench.sum_over_ranks(10.0 * (rank + 1), dist, "cpu")
        q.put((rank, ids, t, n))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_replicas_and_reduce_times():
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ids0, t0, n0), (r1, ids1, t1, n1) = out
    assert not set(ids0) & set(ids1) and len(ids0) == len(ids1) == 3
    assert t0 == t1 == 2.0
    assert n0 == n1 == 30.0
