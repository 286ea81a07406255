"""The N > 1 bench path on CPU: world_size-2 gloo process groups.

bench.py runs replicas only (one graph per rank, no collective on the data
path); what crosses ranks is the slowest rank's time and the job total.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.dist_env()
        t = bench.max_over_ranks(1.0 + 3.0 * rank, dist, "cpu")
        v = bench.job_value(1000, w, bench.max_over_ranks(2.0 + rank, dist, "cpu"))
        # the reference arm: ranks other than 0 leave at once, without output
        class A:
            seed, rhg_log2, warmup, steps = 1, 20, 0, 1
        rc = bench.run_reference(A, r, w) if r != 0 else None
        q.put((rank, r, w, lr, t, v, rc))
    finally:
        dist.destroy_process_group()


def test_two_rank_reductions_gloo():
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
    for rank, r, w, lr, t, v, rc in out:
        assert (r, w, lr) == (rank, 2, rank)
        assert t == 4.0                         # max over ranks
        assert v == pytest.approx(2 * 1000 / 3e-3)  # both ranks' edges over the slowest time
        if rank == 1:
            assert rc == 0


def test_single_process_reductions():
    import bench
    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_value(500, 1, 2.0) == pytest.approx(250000.0)
