"""Seeded synthetic input graphs (inputs only -- none of the min-cut arithmetic).

Both sides of every parity test draw their graphs from here: the CPU oracle
and the CUDA library each receive the same int32 CSR arrays.

Large families come from ``graphgen.cpp`` (OpenMP C++, built with g++ into
``graphgen/_build/libgraphgen.so``); tiny test graphs are built in numpy.

A graph is returned as ``(row_ptr, col, w)``: int32 arrays of a symmetric CSR
with sorted rows, unit or positive integer weights.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.cpp")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u64, i32, f64 = ctypes.c_uint64, ctypes.c_int, ctypes.c_double
            vp = ctypes.c_void_p
            lib.gg_planted.argtypes = [u64, i32, f64, i32]
            lib.gg_rhg.argtypes = [u64, i32, f64, f64]
            lib.gg_rmat_kcore.argtypes = [u64, i32, i32, f64, f64, f64, i32, i32]
            lib.gg_batch.argtypes = [u64, i32, i32, i32, i32, i32, i32]
            for f in ("gg_planted", "gg_rhg", "gg_rmat_kcore", "gg_batch"):
                getattr(lib, f).restype = vp
            lib.gg_n.argtypes = [vp]
            lib.gg_n.restype = i32
            lib.gg_rp_len.argtypes = [vp]
            lib.gg_rp_len.restype = ctypes.c_longlong
            lib.gg_arcs.argtypes = [vp]
            lib.gg_arcs.restype = ctypes.c_longlong
            lib.gg_graphs.argtypes = [vp]
            lib.gg_graphs.restype = i32
            lib.gg_copy.argtypes = [vp, vp, vp, vp, vp, vp]
            lib.gg_free.argtypes = [vp]
            _lib = lib
        return _lib


def _take(h):
    lib = _load()
    try:
        rp = np.empty(lib.gg_rp_len(h), dtype=np.int32)
        m = lib.gg_arcs(h)
        col = np.empty(max(m, 1), dtype=np.int32)
        w = np.empty(max(m, 1), dtype=np.int32)
        G = lib.gg_graphs(h)
        voff = np.empty(G + 1, dtype=np.int64) if G > 0 else None
        aoff = np.empty(G + 1, dtype=np.int64) if G > 0 else None
        lib.gg_copy(h, rp.ctypes.data, col.ctypes.data, w.ctypes.data,
                    voff.ctypes.data if G > 0 else None, aoff.ctypes.data if G > 0 else None)
        col, w = col[:m], w[:m]
        if G > 0:
            return rp, col, w, voff, aoff
        return rp, col, w
    finally:
        lib.gg_free(h)


# ------------------------------------------------------------ large families
def planted(seed: int, block_n: int = 2048, avg_deg: float = 24.0, cross: int = 8):
    """Two G(block_n, avg_deg/(block_n-1)) blocks joined by `cross` random unit
    edges; unit weights (the small plain-method workload)."""
    return _take(_load().gg_planted(seed, block_n, avg_deg, cross))


def rhg(seed: int, n: int = 1 << 20, avg_deg: float = 32.0, gamma: float = 5.0):
    """Threshold random hyperbolic graph, largest connected component, unit
    weights (the paper's synthetic family, Appendix A)."""
    return _take(_load().gg_rhg(seed, n, avg_deg, gamma))


def rmat_kcore(seed: int, scale: int = 22, edge_factor: int = 16, a: float = 0.57,
               b: float = 0.19, c: float = 0.19, k: int = 10, wmax: int = 4):
    """R-MAT, symmetrised and deduplicated, k-core, largest component; weights
    uniform in 1..wmax (stand-in for the paper's real-world k-cores)."""
    return _take(_load().gg_rmat_kcore(seed, scale, edge_factor, a, b, c, k, wmax))


def planted_rhg(seed: int, n_block: int = 1 << 19, avg_deg: float = 32.0, gamma: float = 5.0,
                cross: int = 3):
    """Two threshold RHG graphs (largest components, seeds 2*seed+1 and
    2*seed+2) joined by `cross` distinct random unit edges: a workload of the
    paper's RHG family whose minimum cut (at most `cross`) lies below the
    minimum degree and splits the graph into two large sides.  Vertices of
    the first graph come first; unit weights."""
    ra, ca, _ = rhg(2 * seed + 1, n_block, avg_deg, gamma)
    rb, cb, _ = rhg(2 * seed + 2, n_block, avg_deg, gamma)
    na, nb = len(ra) - 1, len(rb) - 1
    rng = np.random.default_rng([seed, 0x9EC7])
    pairs = set()
    while len(pairs) < cross:
        pairs.add((int(rng.integers(0, na)), int(na + rng.integers(0, nb))))
    cu = np.array(sorted(pairs), dtype=np.int64).reshape(-1, 2)
    cv = cu[np.lexsort((cu[:, 0], cu[:, 1]))]   # the same edges ordered by (v, u)
    src = np.concatenate([np.repeat(np.arange(na), np.diff(ra)), cu[:, 0], cv[:, 1],
                          na + np.repeat(np.arange(nb), np.diff(rb))])
    dst = np.concatenate([ca.astype(np.int64), cu[:, 1], cv[:, 0], na + cb.astype(np.int64)])
    # a stable sort by source keeps each row sorted: in a row of the first
    # graph the cross arcs (to ids >= na) follow its own arcs, in a row of the
    # second they (to ids < na) come first
    order = np.argsort(src, kind="stable")
    n = na + nb
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    col = dst[order].astype(np.int32)
    return np.cumsum(rp).astype(np.int32), col, np.ones(len(col), dtype=np.int32)


def batch(seed: int, G: int = 4096, nmin: int = 50, nmax: int = 2000, dmin: int = 4,
          dmax: int = 16, wmax: int = 100):
    """G connected weighted graphs: returns (row_ptr, col, w, vtx_off, arc_off)
    where graph g's local row_ptr (n_g + 1 entries) starts at
    row_ptr[vtx_off[g] + g] and its arcs at arc_off[g]."""
    return _take(_load().gg_batch(seed, G, nmin, nmax, dmin, dmax, wmax))


def batch_graph(b, g):
    """Graph g of a batch as a standalone (row_ptr, col, w)."""
    rp, col, w, voff, aoff = b
    n = int(voff[g + 1] - voff[g])
    lrp = rp[voff[g] + g: voff[g] + g + n + 1].copy()
    a0, a1 = int(aoff[g]), int(aoff[g + 1])
    return lrp, col[a0:a1].copy(), w[a0:a1].copy()


# ------------------------------------------------------------- tiny graphs
def from_edges(n: int, u, v, w=None):
    """Symmetric CSR with sorted rows from undirected edges (duplicates and
    self-loops are kept as given)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.ones(len(u), dtype=np.int64) if w is None else np.asarray(w, dtype=np.int64)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp)
    return rp.astype(np.int32), dst.astype(np.int32), ww.astype(np.int32)


def complete(n: int, weight: int = 1):
    iu, ju = np.triu_indices(n, 1)
    return from_edges(n, iu, ju, np.full(len(iu), weight))


def cycle(n: int, weight: int = 1):
    u = np.arange(n)
    return from_edges(n, u, (u + 1) % n, np.full(n, weight))


def path_weights(ws):
    n = len(ws) + 1
    u = np.arange(n - 1)
    return from_edges(n, u, u + 1, ws)


def random_tree(n: int, seed: int, wmax: int = 100):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    parent = np.array([perm[rng.integers(0, k)] for k in range(1, n)], dtype=np.int64)
    w = rng.integers(1, wmax + 1, size=n - 1)
    return from_edges(n, perm[1:], parent, w)


def two_cliques(a: int, k: int, seed: int = 0):
    """Two K_a (unit weights) joined by k vertex-disjoint unit edges, k < a-1."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(a, 1)
    u = np.concatenate([iu, iu + a])
    v = np.concatenate([ju, ju + a])
    left = rng.permutation(a)[:k]
    right = rng.permutation(a)[:k] + a
    u = np.concatenate([u, left])
    v = np.concatenate([v, right])
    return from_edges(2 * a, u, v)


def random_gnp(n: int, p: float, seed: int, wmax: int = 100):
    """G(n, p) with weights uniform in 1..wmax (may be disconnected)."""
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    u, v = iu[keep], ju[keep]
    w = rng.integers(1, wmax + 1, size=len(u))
    return from_edges(n, u, v, w)


def random_connected(n: int, extra: int, seed: int, wmax: int = 100):
    """Random spanning tree plus `extra` random (possibly repeated) edges."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    tu = perm[1:]
    tv = np.array([perm[rng.integers(0, k)] for k in range(1, n)], dtype=np.int64)
    eu = rng.integers(0, n, size=extra)
    ev = rng.integers(0, n, size=extra)
    keep = eu != ev
    u = np.concatenate([tu, eu[keep]])
    v = np.concatenate([tv, ev[keep]])
    w = rng.integers(1, wmax + 1, size=len(u))
    return from_edges(n, u, v, w)


def dedupe(rp, col, w):
    """Sum parallel arcs and drop self-loops (the input convention of both the
    oracle and the library), returning a canonical CSR."""
    n = len(rp) - 1
    src = np.repeat(np.arange(n), np.diff(rp))
    keep = src != col
    src, dst, ww = src[keep], col[keep].astype(np.int64), w[keep].astype(np.int64)
    key = src.astype(np.int64) * n + dst
    uniq, inv = np.unique(key, return_inverse=True)
    sw = np.zeros(len(uniq), dtype=np.int64)
    np.add.at(sw, inv, ww)
    s2 = uniq // n
    d2 = uniq % n
    nrp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(nrp, s2 + 1, 1)
    return np.cumsum(nrp).astype(np.int32), d2.astype(np.int32), sw.astype(np.int32)
