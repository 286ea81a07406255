"""The seeded synthetic workloads: the structure each generator promises.

Every generator returns a canonical symmetric CSR (rows strictly increasing,
no self-loops, weights > 0, every arc mirrored with the same weight), is a
pure function of its parameters and seed, and has the shape of the workload
it stands in for (RHG average degree and one component, R-MAT k-core minimum
degree, batch sizes and weights, the planted graph's cross edges)."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components

import graphgen


def canonical_symmetric(rp, col, w):
    n = len(rp) - 1
    rp = np.asarray(rp, dtype=np.int64)
    assert rp[0] == 0 and (np.diff(rp) >= 0).all() and rp[-1] == len(col) == len(w)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert ((col >= 0) & (col < n)).all() and (src != col).all() and (w > 0).all()
    # strictly increasing within each row
    same_row = src[1:] == src[:-1]
    assert (col[1:][same_row] > col[:-1][same_row]).all()
    # mirrored with equal weights: the (u, v, w) and (v, u, w) multisets agree
    fwd = np.stack([src, col, w], 1)
    bwd = np.stack([col, src, w], 1)
    fwd = fwd[np.lexsort(fwd.T[::-1])]
    bwd = bwd[np.lexsort(bwd.T[::-1])]
    assert (fwd == bwd).all()
    return n


def components(rp, col):
    n = len(rp) - 1
    a = csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    return connected_components(a, directed=False)[0]


def test_rhg_shape():
    g = graphgen.rhg(2, 1 << 16, 32.0)
    n = canonical_symmetric(*g)
    assert n == 1 << 16 and components(g[0], g[1]) == 1
    assert abs(len(g[1]) / n - 32.0) < 0.05 * 32.0
    assert (g[2] == 1).all()
    small = graphgen.rhg(1, 1 << 14, 16.0)
    ns = canonical_symmetric(*small)
    assert components(small[0], small[1]) == 1 and ns > (1 << 14) // 4
    assert abs(len(small[1]) / ns - 16.0) < 0.15 * 16.0


def test_rmat_kcore_shape():
    for k in (10, 30):
        g = graphgen.rmat_kcore(3, scale=14, k=k, wmax=4)
        n = canonical_symmetric(*g)
        assert n > 0 and components(g[0], g[1]) == 1
        assert np.diff(g[0]).min() >= k
        assert g[2].min() >= 1 and g[2].max() <= 4


def test_batch_shape():
    b = graphgen.batch(2, G=64, nmin=50, nmax=300, dmin=4, dmax=16, wmax=100)
    rp, col, w, vo, ao = b
    assert len(vo) == len(ao) == 65 and vo[0] == 0 and ao[0] == 0
    for k in range(64):
        g = graphgen.batch_graph(b, k)
        n = canonical_symmetric(*g)
        assert 50 <= n <= 300 and components(g[0], g[1]) == 1
        assert g[2].min() >= 1 and g[2].max() <= 100
        assert 1.9 <= len(g[1]) / n <= 16.5   # spanning tree .. d_max


def test_planted_shape():
    g = graphgen.planted(4, block_n=500, avg_deg=12.0, cross=8)
    n = canonical_symmetric(*g)
    assert n == 1000 and (g[2] == 1).all()
    src = np.repeat(np.arange(n), np.diff(g[0]))
    crossing = (src < 500) != (g[1] < 500)
    assert crossing.sum() == 2 * 8   # both arc directions of the 8 cross edges


@pytest.mark.parametrize("make", [lambda s: graphgen.rhg(s, 1 << 12, 16.0),
                                  lambda s: graphgen.rmat_kcore(s, scale=12, k=5),
                                  lambda s: graphgen.planted(s, block_n=200),
                                  lambda s: graphgen.batch(s, G=8, nmax=100)[:3]])
def test_seeded_and_pure(make):
    a, b, c = make(5), make(5), make(6)
    assert all((x == y).all() for x, y in zip(a, b))
    assert any(len(x) != len(y) or (x != y).any() for x, y in zip(a, c))


def test_batch_lambdas_golden_file():
    # the stored lambdas of the batched workload belong to these very graphs
    # and agree with the oracle on a sample (the benchmark checks every
    # batched result against the file)
    import json
    import os
    import sys
    import oracle
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    sys.path.insert(0, here)
    from make_batch_lambdas import batch_digest
    d = json.load(open(os.path.join(here, "batch_lambdas_seed1.json")))
    b = graphgen.batch(1)
    assert d["arrays_sha256_16"] == batch_digest(b)
    assert len(d["lambdas"]) == len(b[3]) - 1
    for k in range(0, len(b[3]) - 1, 97):
        assert d["lambdas"][k] == oracle.noi(*graphgen.batch_graph(b, k))[0]
