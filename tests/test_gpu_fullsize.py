"""Parity at the workloads' full sizes: lambda bit-exact against the oracle's
sequential NOI and every returned side re-weighed by the oracle.

* R-MAT scale 22, edge factor 16, 10-core, weights 1..4 (the skewed-degree
  plain-path workload);
* RHG n = 2^23, average degree 64, exponent 5 (the learned-bound workload),
  solved with each initial bound;
* planted-cut RHG graphs (two RHG blocks joined by a few unit edges) with
  2^20 and 2^21 vertices, whose minimum cut lies below the minimum degree,
  so the answer must come from a cut the scans or the contractions find
  (Sec. 3.3), not from a trivial cut.
"""
import numpy as np
import pytest

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    import torch
    assert torch.cuda.is_available()
    import paper_1808_05458_gb300 as m
    m.load_library()
    return m


def check(g, res, ref):
    n = len(g[0]) - 1
    side = res.side(n)
    assert res.lam == ref
    assert side[0] == 0 and 0 < side.sum() < n
    assert oracle.cut_weight(*g, side) == ref


def test_rmat_scale22_10core(mc):
    g = graphgen.rmat_kcore(1, scale=22, k=10)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        for order in (mc.MC_PQ_LIFO, mc.MC_PQ_FIFO):
            check(g, G.min_cut(mc.options(pq_order=order)), ref)


def test_rhg_2_23_degree_64_every_bound(mc):
    from paper_1808_05458_gb300 import proposer
    g = graphgen.rhg(1, 1 << 23, 64.0)
    ref, _, _ = oracle.noi(*g)
    P = mc.Proposer.load(proposer.DEFAULT_WEIGHTS)
    with mc.Graph(*g) as G:
        for b in (mc.MC_BOUND_DEGREE, mc.MC_BOUND_LP, mc.MC_BOUND_LEARNED, mc.MC_BOUND_BEST):
            check(g, G.min_cut(mc.options(bound=b, proposer=P.handle)), ref)
    P.close()


@pytest.mark.parametrize("log2n,deg,cross", [(19, 32.0, 3), (20, 64.0, 8)])
def test_planted_cut_below_delta(mc, log2n, deg, cross):
    g = graphgen.planted_rhg(1, 1 << log2n, deg, cross=cross)
    ref, _, _ = oracle.noi(*g)
    assert ref <= cross < int(oracle.degrees(*g).min())
    with mc.Graph(*g) as G:
        for b in (mc.MC_BOUND_DEGREE, mc.MC_BOUND_LP):
            for seed in (1, 2):
                check(g, G.min_cut(mc.options(bound=b, seed=seed)), ref)
