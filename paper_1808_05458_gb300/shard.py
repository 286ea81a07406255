"""Batched solves across ranks, one process per GPU.

The graphs of a batch are independent problems, so a batch shards with no
exchange on the data path: every rank solves a contiguous range of graphs
with one ``mc_batch_min_cut`` call on its own GPU, and the per-graph results
are gathered afterwards.  The ranges split the batch's work (arcs plus
vertices) as evenly as contiguous ranges allow.
"""
import numpy as np


def shard_bounds(vtx_off, arc_off, world: int) -> np.ndarray:
    """Graph bounds per rank: rank r takes graphs [b[r], b[r + 1]).

    The split points are the graph boundaries nearest to equal shares of the
    cumulative work vtx_off + arc_off; ranges are contiguous, cover every
    graph once and may be empty when there are fewer graphs than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = np.asarray(vtx_off, dtype=np.int64) + np.asarray(arc_off, dtype=np.int64)
    G = len(work) - 1
    total = int(work[-1] - work[0])
    b = [0]
    for r in range(1, world):
        target = int(work[0]) + total * r // world
        g = int(np.searchsorted(work, target, side="left"))
        # the nearer of the two boundaries around the target
        if g > 0 and g <= G and target - work[g - 1] < work[min(g, G)] - target:
            g -= 1
        b.append(min(max(g, b[-1]), G))
    b.append(G)
    return np.asarray(b, dtype=np.int64)


def sub_batch(batch, g0: int, g1: int):
    """Graphs [g0, g1) of a concatenated batch (row_ptr, col, w, vtx_off,
    arc_off; graph g's local row_ptr starts at row_ptr[vtx_off[g] + g]) as a
    batch of their own, offsets rebased to 0."""
    rp, col, w, vo, ao = batch
    vo = np.asarray(vo, dtype=np.int64)
    ao = np.asarray(ao, dtype=np.int64)
    return (rp[vo[g0] + g0: vo[g1] + g1], col[ao[g0]: ao[g1]], w[ao[g0]: ao[g1]],
            vo[g0: g1 + 1] - vo[g0], ao[g0: g1 + 1] - ao[g0])


def sharded_batch_min_cut(batch, rank: int, world: int, gather, opts=None, solve=None) -> np.ndarray:
    """lambda of every graph of ``batch``, on every rank.

    This rank solves its range of graphs (``solve(sub_batch)`` returning
    their lambdas; by default one ``mc_batch_min_cut`` call on the current
    GPU) and ``gather(local)`` must return every rank's array in rank order,
    e.g. ``lambda x: (out := [None] * world, dist.all_gather_object(out, x))[0]``."""
    b = shard_bounds(batch[3], batch[4], world)
    g0, g1 = int(b[rank]), int(b[rank + 1])
    if g1 > g0:
        sub = sub_batch(batch, g0, g1)
        if solve is None:
            from .mincut import batch_min_cut
            local = np.asarray(batch_min_cut(*sub, opts=opts)[0], dtype=np.int64)
        else:
            local = np.asarray(solve(sub), dtype=np.int64)
    else:
        local = np.zeros(0, dtype=np.int64)
    parts = gather(local)
    if len(parts) != world:
        raise RuntimeError("gather returned %d parts for %d ranks" % (len(parts), world))
    lam = np.concatenate([np.asarray(p, dtype=np.int64) for p in parts])
    if len(lam) != len(batch[3]) - 1:
        raise RuntimeError("gathered %d results for %d graphs" % (len(lam), len(batch[3]) - 1))
    return lam
