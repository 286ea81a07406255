"""One graph split across ranks (the single-graph multi-GPU layout): each
rank owns a vertex range and scans only its own vertices, lambda-hat is an
all-reduce minimum, the union-find blocks are merged from every rank's
roots, and contracted rows go to their new owners by an all-to-all.

On CPU the process group is gloo with 2 or 3 ranks, and the graph steps are
stand-ins written here: a capped CAPFOREST scan of the rank's own vertices
(every other vertex blacklisted), the oracle's contraction, and the oracle's
exact solve for the last small graph.  The result must be the oracle's
lambda, with a side of that weight.  The GPU test runs the library's
kernels on two ranks that share one GPU (their kernels never wait on one
another: every exchange is a host collective between launches)."""
import heapq
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


class CpuOps:
    """Stand-ins for the graph steps (test code: the oracle is allowed here)."""

    def make(self, n, rp, col, w):
        return (n, np.asarray(rp, np.int64), np.asarray(col, np.int64), np.asarray(w, np.int64))

    def degrees(self, G):
        n, rp, col, w = G
        src = np.repeat(np.arange(n), np.diff(rp))
        d = np.zeros(n, dtype=np.int64)
        np.add.at(d, src, np.where(col != src, w, 0))
        return d

    def scan(self, G, lam, lo, hi):
        # sequential capped scans from the own vertices; a vertex another scan
        # took, or one outside [lo, hi), is blacklisted (left when popped)
        n, rp, col, w = G
        deg = self.degrees(G)
        par = list(range(n))

        def find(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x

        owner = [0] * n
        L, unions, best_side = lam, 0, None
        for s in range(lo, hi):
            if owner[s]:
                continue
            r = {s: 0}
            heap = [(0, s)]
            alpha, scanned, done = 0, [], set()
            while heap:
                _, x = heapq.heappop(heap)
                if x in done:
                    continue
                done.add(x)
                if not (lo <= x < hi) or owner[x]:
                    continue
                owner[x] = s + 1
                scanned.append(x)
                alpha += deg[x] - 2 * r.get(x, 0)
                if len(scanned) < n and alpha < L:
                    L = alpha
                    best_side = list(scanned)
                for a in range(rp[x], rp[x + 1]):
                    y, c = int(col[a]), int(w[a])
                    if y == x or y in done:
                        continue
                    ry = r.get(y, 0)
                    if ry < L <= ry + c:
                        a_, b_ = find(x), find(y)
                        if a_ != b_:
                            par[max(a_, b_)] = min(a_, b_)
                            unions += 1
                    r[y] = ry + c
                    heapq.heappush(heap, (-min(r[y], L), y))
        lab = np.array([find(v) for v in range(n)], dtype=np.int32)
        bits = np.zeros(n, dtype=np.uint8)
        if best_side is not None:
            bits[best_side] = 1
        words = np.packbits(bits, bitorder="little")
        words = np.concatenate([words, np.zeros((-len(words)) % 4, np.uint8)]).view(np.uint32)
        return lab, L, unions, words

    def contract(self, G, lab, nc, clamp):
        import oracle
        n, rp, col, w = G
        crp, ccol, cw = oracle.contract(rp.astype(np.int32), col.astype(np.int32), w.astype(np.int32),
                                        np.asarray(lab, np.int32), nc)
        return crp, ccol, np.minimum(cw, clamp)

    def solve(self, n, rp, col, w):
        import oracle
        lam, side, _ = oracle.noi(rp, col, w)
        return lam, side

    def close(self, G):
        pass


def _graphs():
    import graphgen
    rng = np.random.default_rng(5)
    out = [graphgen.random_connected(int(rng.integers(20, 60)), int(rng.integers(30, 200)), seed=i, wmax=9)
           for i in range(6)]
    out += [graphgen.planted(3, block_n=60, avg_deg=8, cross=2), graphgen.rhg(2, 300, 10.0),
            graphgen.two_cliques(12, 3, seed=1), graphgen.cycle(40, 2),
            graphgen.from_edges(30, np.r_[np.arange(14), np.arange(15, 29)],
                                np.r_[np.arange(1, 15), np.arange(16, 30)], np.full(28, 3))]
    return out


def _split(g, rank, world):
    from paper_1808_05458_gb300 import dist
    rp, col, w = g
    n = len(rp) - 1
    b = dist.owner_bounds(n, world)
    lo, hi = int(b[rank]), int(b[rank + 1])
    a0, a1 = rp[lo], rp[hi]
    return n, rp[lo:hi + 1] - a0, col[a0:a1], w[a0:a1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, use_gpu, q):
    import torch.distributed as dist
    from paper_1808_05458_gb300 import dist as sg
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = sg.TorchComm(dist)
        if use_gpu:
            import torch
            torch.cuda.set_device(0)
            ops, small = sg.LibraryOps(), 64
        else:
            ops, small = CpuOps(), 2
        res = []
        try:
            for g in (_graphs() if not use_gpu else _gpu_graphs()):
                n, rp, col, w = _split(g, rank, world)
                lam, side = sg.min_cut(comm, n, rp, col, w, ops=ops, small=small)
                res.append((int(lam), side))
        except Exception as e:  # report at once instead of leaving the parent waiting
            q.put((rank, repr(e)))
            raise
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def _run(world, use_gpu=False, graphs=None):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, use_gpu, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(world):
        r, res = q.get(timeout=600)
        assert not isinstance(res, str), f"rank {r}: {res}"
        out[r] = res
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def _check(out, graphs, world):
    import oracle
    for k, g in enumerate(graphs):
        ref = oracle.noi(*g)[0]
        n = len(g[0]) - 1
        for r in range(world):
            lam, side = out[r][k]
            assert lam == ref, (k, r, lam, ref)
            assert side[0] == 0 and 0 < side.sum() < n
            assert oracle.cut_weight(*g, side) == ref
        for r in range(1, world):
            assert (out[r][k][1] == out[0][k][1]).all()


def test_merge_labels_joins_partitions():
    from paper_1808_05458_gb300 import dist
    a = np.array([0, 0, 2, 2, 4, 5, 5], dtype=np.int32)   # {0,1} {2,3} {4} {5,6}
    b = np.array([0, 1, 1, 3, 3, 5, 6], dtype=np.int32)   # {1,2} {3,4}
    assert list(dist.merge_labels([a, b], 7)) == [0, 0, 0, 0, 0, 5, 5]
    rng = np.random.default_rng(1)
    for _ in range(50):
        n = int(rng.integers(2, 40))
        parts = []
        for _ in range(3):
            p = np.arange(n)
            for u, v in rng.integers(0, n, size=(int(rng.integers(0, n)), 2)):
                ru, rv = p[u], p[v]
                p[p == max(ru, rv)] = min(ru, rv)
            parts.append(p.astype(np.int32))
        got = dist.merge_labels(parts, n)
        # brute force: components of the union of the partitions
        comp = np.arange(n)
        changed = True
        while changed:
            changed = False
            for p in parts:
                for v in range(n):
                    m = min(comp[v], comp[p[v]])
                    if comp[v] != m or comp[p[v]] != m:
                        comp[v] = comp[p[v]] = m
                        changed = True
        for v in range(n):
            comp[v] = comp[comp[v]]
        assert (got == comp).all()


def test_owner_bounds():
    from paper_1808_05458_gb300 import dist
    for n, world in ((10, 3), (2, 2), (7, 1), (100, 8)):
        b = dist.owner_bounds(n, world)
        assert b[0] == 0 and b[-1] == n and (np.diff(b) >= 0).all() and np.ptp(np.diff(b)) <= 1


@pytest.mark.parametrize("world", [1, 2, 3])
def test_single_graph_split_on_cpu(world):
    out = _run(world)
    _check(out, _graphs(), world)


def _gpu_graphs():
    import graphgen
    return [graphgen.planted(2), graphgen.rhg(3, 1 << 14, 24.0),
            graphgen.planted_rhg(2, 1 << 12, 32.0, cross=3), graphgen.rmat_kcore(1, scale=14, k=8)]


@pytest.mark.gpu
def test_single_graph_split_on_gpu():
    out = _run(2, use_gpu=True)
    _check(out, _gpu_graphs(), 2)
