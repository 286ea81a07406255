"""One graph across ranks, one process per GPU (the single-graph split of the
exact loop, Alg. 2).

Every rank owns a contiguous range of the current graph's vertices and holds
their rows (the neighbours are global ids).  A round:

* each rank runs the concurrent capped CAPFOREST scans on its own vertices
  only (``mc_step_capforest_range``): every other vertex counts as
  blacklisted (Sec. 3.2, Lemma 2 part 3), so it still gathers r-values and
  can be united, but is never scanned;
* lambda-hat is the minimum over the ranks (an all-reduce), and the rank
  whose scan lowered it most sends the side of that cut (Sec. 3.3);
* the ranks' union-find blocks are merged: every rank's root array is
  gathered and the blocks of all of them are joined (pointer jumping), which
  numbers the contracted vertices the same way on every rank;
* each rank contracts its own rows by the merged labels
  (``mc_step_contract``, weights clamped to lambda-hat) and sends every
  contracted row to the rank that owns the row's new vertex (an all-to-all);
  the receiver sums the parallel arcs that came from several ranks and
  clamps the sums to lambda-hat;
* lambda-hat = min(lambda-hat, minimum degree) over the ranks.

When a round unites nothing, or the graph has shrunk to ``small`` vertices,
the rows are gathered on rank 0, which finishes with the exact single-GPU
solve (the multi-GPU stand-in for Alg. 2's full-scan fallback) and sends the
result to every rank.

The steps that touch the graph run through ``ops`` (by default the library's
CUDA kernels on the current GPU); the collectives run through ``comm``.
"""
from __future__ import annotations

import numpy as np


def owner_bounds(n: int, world: int) -> np.ndarray:
    """Vertex bounds per rank: rank r owns [b[r], b[r + 1]) (equal split)."""
    return (np.arange(world + 1, dtype=np.int64) * n) // world


class TorchComm:
    """The collectives of the split over a torch.distributed process group
    (gloo carries host arrays; every payload here is a numpy array or a
    scalar)."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def _gather_objects(self, x):
        out = [None] * self.world
        self.dist.all_gather_object(out, x, group=self.group)
        return out

    def allreduce_min(self, x: int) -> int:
        return int(min(self._gather_objects(int(x))))

    def allreduce_sum(self, x: int) -> int:
        return int(sum(self._gather_objects(int(x))))

    def all_gather(self, a):
        return self._gather_objects(a)

    def all_to_all(self, parts):
        # parts[d] goes to rank d; returns what every rank sent to this one
        everything = self._gather_objects(parts)
        return [everything[s][self.rank] for s in range(self.world)]

    def broadcast(self, x, root: int):
        box = [x]
        self.dist.broadcast_object_list(box, src=root, group=self.group)
        return box[0]


class LibraryOps:
    """The graph steps in the library's CUDA kernels (current GPU)."""

    def __init__(self, opts=None):
        from . import mincut
        self.mc = mincut
        self.opts = opts

    def make(self, n, rp, col, w):
        # rows of the other ranks' vertices are empty: not symmetric by design
        return self.mc.Graph(rp, col, w, trust=True)

    def scan(self, G, lam, lo, hi):
        return G.capforest_range(int(lam), int(lo), int(hi), self.opts)

    def degrees(self, G):
        return G.degrees()

    def contract(self, G, lab, nc, clamp):
        return G.contract(lab, nc, clamp)

    def solve(self, n, rp, col, w):
        with self.mc.Graph(rp, col, w) as G:
            res = G.min_cut(self.opts)
            return res.lam, res.side(n)

    def close(self, G):
        G.close()


def _rows_to_csr(n, src, dst, w):
    """CSR over n vertices of the arcs (src, dst, w), rows in source order
    (the graph build sorts and merges each row)."""
    order = np.argsort(src, kind="stable")
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, np.asarray(src, dtype=np.int64) + 1, 1)
    return (np.cumsum(rp).astype(np.int32), np.asarray(dst)[order].astype(np.int32),
            np.asarray(w)[order].astype(np.int32))


def merge_received(n, src, dst, w, clamp):
    """Parallel arcs that came from several ranks summed and clamped to
    lambda-hat.  Each sender clamped its own part, so only the clamp of the
    sum gives both directions of an edge the same weight, min(c, lambda-hat),
    which keeps every degree and every scan's alpha exact below the bound."""
    key = np.asarray(src, dtype=np.int64) * n + np.asarray(dst, dtype=np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    tot = np.zeros(len(uk), dtype=np.int64)
    np.add.at(tot, inv, np.asarray(w, dtype=np.int64))
    return uk // n, uk % n, np.minimum(tot, clamp)


def merge_labels(parts, n: int) -> np.ndarray:
    """The blocks of several partitions of [0, n) joined: parts[r][v] is the
    smallest vertex of v's block in partition r; the result maps v to the
    smallest vertex of its joined block."""
    lab = np.arange(n, dtype=np.int64)
    while True:
        prev = lab.copy()
        for p in parts:
            p = np.asarray(p, dtype=np.int64)
            m = np.minimum(lab, lab[p])
            np.minimum.at(m, p, m)       # a root takes its members' smallest label
            lab = np.minimum(lab, m[p])  # and every member the root's
            lab = np.minimum(lab, m)
        while True:                      # pointer jumping to the fixed point
            nxt = lab[lab]
            if (nxt == lab).all():
                break
            lab = nxt
        if (lab == prev).all():
            return lab


def _canonical(side):
    side = np.asarray(side, dtype=np.uint8)
    return 1 - side if side[0] else side


def min_cut(comm, n0: int, rp_own, col_own, w_own, ops=None, small: int = 4096, max_rounds: int = 10_000):
    """lambda and one minimum-cut side (uint8 array over the n0 vertices, 1 =
    not vertex 0's side) of the graph whose rows of the vertices
    owner_bounds(n0, world)[rank] .. [rank + 1] this rank holds: rp_own has
    (own vertex count + 1) offsets, col_own global neighbour ids.  The same
    result is returned on every rank."""
    ops = ops or LibraryOps()
    rank, world = comm.rank, comm.world
    b = owner_bounds(n0, world)
    lo = int(b[rank])
    own_n = int(b[rank + 1]) - lo
    rp_own = np.asarray(rp_own, dtype=np.int64)
    src = lo + np.repeat(np.arange(own_n, dtype=np.int64), np.diff(rp_own))
    dst = np.asarray(col_own, dtype=np.int64)
    wt = np.asarray(w_own, dtype=np.int64)
    n = n0
    orig = np.arange(n0, dtype=np.int64)          # original vertex -> current vertex

    def degree_bound(G, lo, hi):
        d = ops.degrees(G)[lo:hi]
        dmin = int(d.min()) if len(d) else np.iinfo(np.int64).max
        gmin = comm.allreduce_min(dmin)
        arg = int(lo + np.argmin(d)) if len(d) and dmin == gmin else n
        return gmin, comm.allreduce_min(arg)

    def finish_on_rank0(lam, side):
        parts = comm.all_gather((src, dst, wt))
        res = None
        if rank == 0:
            s = np.concatenate([p[0] for p in parts])
            d = np.concatenate([p[1] for p in parts])
            w = np.concatenate([p[2] for p in parts])
            res = ops.solve(n, *_rows_to_csr(n, s, d, w)) if n >= 2 else (lam, None)
        res = comm.broadcast(res, 0)
        if res[0] < lam:
            return int(res[0]), np.asarray(res[1], dtype=np.uint8)[orig]
        return lam, side

    lam, side = None, None
    for _ in range(max_rounds):
        b = owner_bounds(n, world)
        lo, hi = int(b[rank]), int(b[rank + 1])
        if n < 2:
            break
        G = ops.make(n, *_rows_to_csr(n, src, dst, wt))
        dmin, arg = degree_bound(G, lo, hi)
        if lam is None or dmin < lam:
            lam = dmin
            side = (orig == arg).astype(np.uint8)
        if lam == 0 or n <= small:
            ops.close(G)
            lam, side = finish_on_rank0(lam, side) if lam > 0 else (lam, side)
            return lam, _canonical(side)
        lab, lam_r, unions, bits = ops.scan(G, lam, lo, hi)
        lam_new = comm.allreduce_min(lam_r)
        if lam_new < lam:
            winner = comm.allreduce_min(rank if lam_r == lam_new else world)
            bits = comm.broadcast(bits if rank == winner else None, winner)
            cur = np.unpackbits(np.asarray(bits, dtype=np.uint32).view(np.uint8), bitorder="little")[:n]
            lam, side = lam_new, cur[orig].astype(np.uint8)
        merged = merge_labels(comm.all_gather(lab), n)
        roots, new_id = np.unique(merged, return_inverse=True)
        nc = len(roots)
        if nc == n:
            # no rank united anything: the exact solve of the whole graph
            ops.close(G)
            lam, side = finish_on_rank0(lam, side)
            return lam, _canonical(side)
        crp, ccol, cw = ops.contract(G, new_id.astype(np.int32), nc, lam)
        ops.close(G)
        orig = new_id[orig]
        # every contracted row goes to the owner of its new vertex
        csrc = np.repeat(np.arange(nc, dtype=np.int64), np.diff(np.asarray(crp, dtype=np.int64)))
        nb = owner_bounds(nc, world)
        dest = np.searchsorted(nb, csrc, side="right") - 1
        parts = [(csrc[dest == d], np.asarray(ccol)[dest == d], np.asarray(cw)[dest == d]) for d in range(world)]
        recv = comm.all_to_all(parts)
        src, dst, wt = merge_received(nc, np.concatenate([p[0] for p in recv]),
                                      np.concatenate([p[1] for p in recv]),
                                      np.concatenate([p[2] for p in recv]), lam)
        n = nc
    return lam, _canonical(side)
