"""Batched solves across ranks on CPU: the graph split and the gather, with
world_size-2 gloo process groups (the per-graph solve is the oracle here;
on GPUs it is one mc_batch_min_cut call per rank)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _oracle_solve(sub):
    import graphgen
    import oracle
    G = len(sub[3]) - 1
    return [oracle.noi(*graphgen.batch_graph(sub, g))[0] for g in range(G)]


@pytest.mark.parametrize("world", [1, 2, 3, 8, 200])
def test_shard_bounds_cover_and_balance(world):
    import graphgen
    from paper_1808_05458_gb300 import shard
    b = graphgen.batch(3, G=97, nmin=20, nmax=300)
    vo, ao = np.asarray(b[3]), np.asarray(b[4])
    bounds = shard.shard_bounds(vo, ao, world)
    assert len(bounds) == world + 1 and bounds[0] == 0 and bounds[-1] == 97
    assert (np.diff(bounds) >= 0).all()
    work = vo + ao
    per_graph = np.diff(work)
    shares = work[bounds[1:]] - work[bounds[:-1]]
    assert shares.sum() == work[-1]
    # every rank is within one graph's work of an even share
    assert (np.abs(shares - work[-1] / world) <= per_graph.max()).all()


def test_sub_batch_is_the_same_graphs():
    import graphgen
    from paper_1808_05458_gb300 import shard
    b = graphgen.batch(4, G=12, nmin=10, nmax=60)
    sub = shard.sub_batch(b, 5, 9)
    for k in range(4):
        a, c = graphgen.batch_graph(b, 5 + k), graphgen.batch_graph(sub, k)
        assert all((x == y).all() for x, y in zip(a, c))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import graphgen
    from paper_1808_05458_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = graphgen.batch(5, G=23, nmin=10, nmax=80)

        def gather(x):
            out = [None] * world
            dist.all_gather_object(out, x)
            return out

        lam = shard.sharded_batch_min_cut(b, rank, world, gather, solve=_oracle_solve)
        q.put((rank, lam.tolist()))
    finally:
        dist.destroy_process_group()


def test_two_rank_batch_gloo():
    import torch.multiprocessing as mp
    import graphgen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = _oracle_solve(graphgen.batch(5, G=23, nmin=10, nmax=80))
    for rank, lam in out:
        assert lam == ref
