"""The benchmark's multi-replica harness on CPU (gloo, world size 2).

The single-pair path does not shard, so `bench.py --gpus N` runs N independent
replicas and no collective touches the data path.  What does run across ranks
is the timing: the job time is the slowest replica's, and the whole-job value
counts every replica's cells.  Both are checked here with two gloo ranks.
"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank                      # rank 1 is the slow replica
        total = bench._max_over_ranks(dist, mine, "cpu")
        q.put((rank, total, bench._job_gcups(world, 1_000_000, 2, total)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value():
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
    assert [o[1] for o in out] == [15.0, 15.0]
    # two replicas x 2 steps x 1e6 cells in 15 s
    assert out[0][2] == pytest.approx(2 * 2 * 1e6 / 15.0 / 1e9)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(None, 3.5, "cpu") == 3.5
    assert bench._job_gcups(1, 10 ** 9, 1, 1.0) == 1.0
