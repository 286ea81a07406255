"""Pins for the CPU oracle against things other than itself.

Each test fixes the oracle to a value that the paper's definitions or the
mathematics determine independently:

* hand-derived cut capacities and minimum cuts (tests/golden/tiny_cuts.json,
  Sec. 2.1 definitions);
* closed forms of lambda for K_n, C_n, trees, two cliques joined by k
  disjoint edges, disconnected graphs;
* brute-force enumeration (definition of lambda, Sec. 2.1) against
  Stoer-Wagner and NOI on thousands of random tiny graphs;
* Lemma 1 (capped queue) -- capped and uncapped NOI agree;
* contraction (Sec. 2.1) preserves the capacity of every cut that keeps each
  block on one side;
* the published splitmix64 output sequence for seed 1234567;
* hand-derived Padberg-Rinaldi blocks where PR2 and PR3 must fire (and
  where a one-sided or max-degree variant would not), and hand-derived
  label-propagation sweeps where synchronous half-sweeps, the parity split
  and the weighted choice each give a different result from the obvious
  alternative.
"""
import json
import os

import numpy as np
import pytest

import graphgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def side_ok(side, n):
    s = np.asarray(side)
    return len(s) == n and s[0] == 0 and 0 < s.sum() < n


def test_splitmix64_published_sequence():
    # Vigna's reference splitmix64: state advances by the golden gamma and each
    # output is the finaliser of the new state; seed 1234567 gives these five.
    expected = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                4593380528125082431, 16408922859458223821]
    state = 1234567
    got = []
    for _ in range(5):
        got.append(oracle.splitmix64(state))
        state = (state + 0x9E3779B97F4A7C15) % 2**64
    assert got == expected


@pytest.mark.parametrize("case", json.load(open(os.path.join(GOLDEN, "tiny_cuts.json")))["cases"],
                         ids=lambda c: c["name"])
def test_golden_tiny_cuts(case):
    n = case["n"]
    e = np.array(case["edges"])
    g = graphgen.from_edges(n, e[:, 0], e[:, 1], e[:, 2])
    side = np.zeros(n, dtype=np.uint8)
    side[case["side"]] = 1
    assert oracle.cut_weight(*g, side) == case["side_capacity"]
    assert oracle.cut_weight(*g, 1 - side) == case["side_capacity"]
    for algo in (oracle.brute_force, oracle.stoer_wagner):
        lam, s = algo(*g)
        assert lam == case["lambda"]
        assert side_ok(s, n) and oracle.cut_weight(*g, s) == lam
    lam, s, _ = oracle.noi(*g)
    assert lam == case["lambda"] and oracle.cut_weight(*g, s) == lam


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 11])
@pytest.mark.parametrize("wt", [1, 7])
def test_complete_graph(n, wt):
    g = graphgen.complete(n, wt)
    expect = (n - 1) * wt
    assert oracle.brute_force(*g)[0] == expect
    assert oracle.stoer_wagner(*g)[0] == expect
    assert oracle.noi(*g)[0] == expect
    assert oracle.noi(*g, capped=False)[0] == expect


@pytest.mark.parametrize("n", [3, 4, 9, 16])
@pytest.mark.parametrize("wt", [1, 5])
def test_cycle(n, wt):
    g = graphgen.cycle(n, wt)
    expect = 2 * wt
    if n <= 20:
        assert oracle.brute_force(*g)[0] == expect
    assert oracle.stoer_wagner(*g)[0] == expect
    assert oracle.noi(*g)[0] == expect


@pytest.mark.parametrize("seed", range(6))
def test_tree_is_min_edge(seed):
    g = graphgen.random_tree(14, seed)
    expect = int(g[2].min())
    assert oracle.brute_force(*g)[0] == expect
    assert oracle.stoer_wagner(*g)[0] == expect
    lam, side, _ = oracle.noi(*g)
    assert lam == expect and oracle.cut_weight(*g, side) == expect


@pytest.mark.parametrize("a,k", [(5, 1), (6, 3), (8, 2), (30, 5)])
def test_two_cliques(a, k):
    g = graphgen.two_cliques(a, k, seed=a + k)
    if 2 * a <= 20:
        assert oracle.brute_force(*g)[0] == k
    lam, side = oracle.stoer_wagner(*g)
    assert lam == k
    # the only cut of weight k separates the cliques
    assert side[:a].sum() in (0, a) and side[a:].sum() in (0, a)
    assert oracle.noi(*g)[0] == k


def test_disconnected_is_zero():
    u = np.array([0, 1, 3, 4])
    v = np.array([1, 2, 4, 5])
    g = graphgen.from_edges(6, u, v, np.array([3, 4, 5, 6]))
    assert oracle.brute_force(*g)[0] == 0
    lam, side = oracle.stoer_wagner(*g)
    assert lam == 0 and oracle.cut_weight(*g, side) == 0
    lam, side, _ = oracle.noi(*g)
    assert lam == 0 and oracle.cut_weight(*g, side) == 0 and side_ok(side, 6)


def test_isolated_vertex_is_zero():
    g = graphgen.from_edges(4, np.array([0, 1]), np.array([1, 2]))
    assert oracle.brute_force(*g)[0] == 0
    assert oracle.stoer_wagner(*g)[0] == 0
    assert oracle.noi(*g)[0] == 0


def _random_tiny(rng, i):
    n = int(rng.integers(2, 15))
    kind = i % 4
    if kind == 0:
        g = graphgen.random_gnp(n, float(rng.uniform(0.15, 0.9)), seed=i, wmax=100)
    elif kind == 1:
        g = graphgen.random_gnp(n, float(rng.uniform(0.3, 1.0)), seed=i, wmax=3)
    elif kind == 2:
        g = graphgen.random_connected(n, int(rng.integers(0, 3 * n)), seed=i, wmax=10)
    else:
        # parallel arcs and self-loops in the input
        m = int(rng.integers(1, 3 * n))
        u = rng.integers(0, n, size=m)
        v = rng.integers(0, n, size=m)
        g = graphgen.from_edges(n, u, v, rng.integers(1, 6, size=m))
    return n, g


def test_random_tiny_all_agree():
    rng = np.random.default_rng(12345)
    for i in range(2500):
        n, g = _random_tiny(rng, i)
        bf, sbf = oracle.brute_force(*g)
        sw, ssw = oracle.stoer_wagner(*g)
        noi, snoi, _ = oracle.noi(*g, seed=i)
        noi_u, _, _ = oracle.noi(*g, capped=False, seed=i + 1)
        assert bf == sw == noi == noi_u, (i, bf, sw, noi, noi_u)
        for s in (sbf, ssw, snoi):
            assert side_ok(s, n)
            assert oracle.cut_weight(*g, s) == bf


def test_noi_medium_seeds_and_cap():
    # Lemma 1: capping the queue at lambda-hat keeps lambda; the start vertex
    # (Alg. 3 "insert random vertex") does not change lambda either.
    for i in range(12):
        g = graphgen.random_connected(300 + 50 * i, 900 + 100 * i, seed=100 + i, wmax=20)
        ref = oracle.stoer_wagner(*g)[0]
        for seed in range(3):
            lam, side, _ = oracle.noi(*g, capped=bool(seed % 2), seed=seed)
            assert lam == ref
            assert oracle.cut_weight(*g, side) == ref


def test_planted_small_block_graph():
    g = graphgen.planted(3, block_n=300, avg_deg=12, cross=3)
    n = len(g[0]) - 1
    deg = oracle.degrees(*g)
    ref, side = oracle.stoer_wagner(*g)
    assert ref <= min(3, int(deg.min()))
    lam, s, _ = oracle.noi(*g)
    assert lam == ref and oracle.cut_weight(*g, s) == ref and side_ok(s, n)


def test_degrees_closed_forms():
    g = graphgen.complete(7, 3)
    assert (oracle.degrees(*g) == 18).all()
    g = graphgen.from_edges(3, np.array([0, 0, 1, 2]), np.array([1, 1, 2, 2]),
                            np.array([2, 3, 4, 50]))
    assert list(oracle.degrees(*g)) == [5, 9, 4]


def _rand_labels(rng, n):
    nc = int(rng.integers(1, n + 1))
    lab = rng.integers(0, nc, size=n)
    lab[rng.permutation(n)[:nc]] = np.arange(nc)  # every block non-empty
    return lab.astype(np.int32), nc


def test_contract_preserves_block_respecting_cuts():
    rng = np.random.default_rng(7)
    for i in range(300):
        n, g = _random_tiny(rng, i)
        lab, nc = _rand_labels(rng, n)
        crp, ccol, cw = oracle.contract(*g, lab, nc)
        # canonical: sorted rows, no self-loops, no zero weights
        for b in range(nc):
            row = ccol[crp[b]:crp[b + 1]]
            assert (np.diff(row) > 0).all() and (row != b).all()
        assert (cw > 0).all()
        # total weight: all arcs minus those inside blocks
        rp, col, w = g
        src = np.repeat(np.arange(n), np.diff(rp))
        cross = lab[src] != lab[col]
        assert cw.sum() == w[cross].astype(np.int64).sum()
        # every cut of the contracted graph weighs what its preimage weighs
        for _ in range(4):
            a = rng.integers(0, 2, size=nc).astype(np.uint8)
            pre = a[lab]
            c_sum = 0
            csrc = np.repeat(np.arange(nc), np.diff(crp))
            c_sum = int(cw[a[csrc] != a[ccol]].sum()) // 2
            assert c_sum == oracle.cut_weight(*g, pre)


def test_label_prop_cliques_converge_to_min_id():
    # two disjoint cliques: labels only travel along edges and each clique
    # settles on one label, the smallest id in it
    iu, ju = np.triu_indices(6, 1)
    u = np.concatenate([iu, iu + 6])
    v = np.concatenate([ju, ju + 6])
    g = graphgen.from_edges(12, u, v)
    for seed in range(5):
        lab = oracle.label_prop(*g, iters=6, seed=seed)
        assert (lab[:6] == 0).all() and (lab[6:] == 6).all()


def test_label_prop_labels_stay_in_component():
    rng = np.random.default_rng(3)
    for i in range(50):
        n, g = _random_tiny(rng, i)
        lab = oracle.label_prop(*g, iters=3, seed=i)
        # component of each vertex via brute BFS
        rp, col, _ = g
        comp = -np.ones(n, dtype=np.int64)
        for s in range(n):
            if comp[s] >= 0:
                continue
            stack = [s]
            comp[s] = s
            while stack:
                x = stack.pop()
                for y in col[rp[x]:rp[x + 1]]:
                    if comp[y] < 0:
                        comp[y] = s
                        stack.append(y)
        assert (comp[lab] == comp).all()
        # zero sweeps leave the identity labelling
        assert (oracle.label_prop(*g, iters=0, seed=i) == np.arange(n)).all()


def test_pr_tests_preserve_lambda():
    # every PR contraction keeps min(lambda-hat, lambda(G / PR)) = lambda(G)
    rng = np.random.default_rng(11)
    checked = 0
    for i in range(600):
        n, g = _random_tiny(rng, i)
        if n < 3:
            continue
        lam = oracle.brute_force(*g)[0]
        deg = oracle.degrees(*g)
        for bound in (int(deg.min()), max(lam, int(deg.min()) - 1), lam):
            if bound < lam:
                continue
            for level in (1, 2, 3, 4):
                lab = oracle.pr_tests(*g, bound, level)
                roots, lab2 = np.unique(lab, return_inverse=True)
                nc = len(roots)
                if nc == 1:
                    assert bound == lam
                    continue
                crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), nc)
                lam_c = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))[0]
                assert min(bound, lam_c) == lam, (i, level, bound, lam, lam_c)
                checked += 1
    assert checked > 1000


def test_pr2_strictness_chain():
    # two K_10 joined by a path x - u1 - u2 - y of unit edges: lambda = 1,
    # delta = 2.  "2c >= min d" would hold on every path edge and contracting
    # them all at once would lose the cut of weight 1; the strict test keeps it.
    a = 10
    iu, ju = np.triu_indices(a, 1)
    u = np.concatenate([iu, iu + a, [0, 2 * a, 2 * a + 1]])
    v = np.concatenate([ju, ju + a, [2 * a, 2 * a + 1, a]])
    g = graphgen.from_edges(2 * a + 2, u, v)
    assert oracle.stoer_wagner(*g)[0] == 1
    lab = oracle.pr_tests(*g, 2, 2)
    roots, lab2 = np.unique(lab, return_inverse=True)
    crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
    assert oracle.stoer_wagner(crp.astype(np.int32), ccol, cw.astype(np.int32))[0] == 1


def test_pr1_pr4_closed_forms():
    # PR1: an edge of weight >= bound is always merged.
    g = graphgen.from_edges(4, np.array([0, 1, 2]), np.array([1, 2, 3]), np.array([5, 1, 5]))
    lab = oracle.pr_tests(*g, 5, 1)
    assert lab[0] == lab[1] and lab[2] == lab[3] and lab[1] != lab[2]
    # PR4 on K_n: c(u,v) + (n - 2) two-hop paths = n - 1 >= bound n - 1.
    g = graphgen.complete(6)
    lab = oracle.pr_tests(*g, 5, 4)
    assert (lab == 0).all()
    assert len(np.unique(oracle.pr_tests(*g, 5, 3))) == 6  # PR3 needs > d/2


def _blocks_safe(g, lab, bound):
    # min(bound, lambda(G / blocks)) = lambda(G): the test's unions are safe
    lam = oracle.brute_force(*g)[0]
    roots, lab2 = np.unique(lab, return_inverse=True)
    if len(roots) == 1:
        return bound == lam
    crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
    lam_c = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))[0]
    return min(bound, lam_c) == lam


def test_pr2_fires_on_heavy_edges():
    # Edges (weight): 0-1 (5), 0-2 (4), 1-2 (4), 1-3 (3), 2-3 (6).
    # Weighted degrees: d0 = 9, d1 = 12, d2 = 14, d3 = 9; delta = bound = 9,
    # so PR1 (c >= 9) passes nothing and no vertex has two equal-weight arcs
    # as its only ones (the degree-2 rule stays out).
    # PR2, 2c > min(d(u), d(v)):
    #   0-1: 10 > min(9, 12) = 9   passes (but 10 <= max = 12)
    #   0-2:  8 > min(9, 14) = 9   fails
    #   1-2:  8 > min(12, 14) = 12 fails
    #   1-3:  6 > min(12, 9) = 9   fails
    #   2-3: 12 > min(14, 9) = 9   passes (but 12 <= max = 14)
    # Blocks {0, 1} and {2, 3}: labels (smallest member) 0, 0, 2, 2.
    u = np.array([0, 0, 1, 1, 2])
    v = np.array([1, 2, 2, 3, 3])
    c = np.array([5, 4, 4, 3, 6])
    g = graphgen.from_edges(4, u, v, c)
    assert list(oracle.degrees(*g)) == [9, 12, 14, 9]
    assert list(oracle.pr_tests(*g, 9, 1)) == [0, 1, 2, 3]
    lab = oracle.pr_tests(*g, 9, 2)
    assert list(lab) == [0, 0, 2, 2]
    assert _blocks_safe(g, lab, 9)


def test_pr3_fires_on_a_triangle_meeting_both_conditions():
    # Prism: triangles {0, 1, 2} and {3, 4, 5} with edges of weight 3, rungs
    # 0-3 (5), 1-4 (6), 2-5 (5).  d = 11, 12, 11, 11, 12, 11; bound = delta
    # = 11.  PR1 (c >= 11) and PR2 (2c > min d: triangle 6 > 11, rungs
    # 10 > 11, 12 > 12, 10 > 11) pass nothing; every vertex has three arcs.
    # PR3 for edge {u, v} with common neighbour w needs
    # 2(c(u,v) + c(u,w)) > d(u) and 2(c(u,v) + c(v,w)) > d(v):
    #   0-2 (w = 1): 12 > d0 = 11 and 12 > d2 = 11          passes
    #   0-1 (w = 2): 12 > d0 = 11 but 12 > d1 = 12 is false  fails
    #   1-2 (w = 0): 12 > d1 = 12 is false                   fails
    # and the same in the second triangle (3-5 passes); rungs have no common
    # neighbour.  PR4 (level 4): c + min over the common neighbour = 3 + 3
    # = 6 < 11 on every triangle edge, so level 4 adds nothing.
    # Blocks {0, 2}, {1}, {3, 5}, {4}: labels 0, 1, 0, 3, 4, 3.
    u = np.array([0, 0, 1, 3, 3, 4, 0, 1, 2])
    v = np.array([1, 2, 2, 4, 5, 5, 3, 4, 5])
    c = np.array([3, 3, 3, 3, 3, 3, 5, 6, 5])
    g = graphgen.from_edges(6, u, v, c)
    assert list(oracle.degrees(*g)) == [11, 12, 11, 11, 12, 11]
    assert list(oracle.pr_tests(*g, 11, 2)) == [0, 1, 2, 3, 4, 5]
    for level in (3, 4):
        lab = oracle.pr_tests(*g, 11, level)
        assert list(lab) == [0, 1, 0, 3, 4, 3], level
        assert _blocks_safe(g, lab, 11)


def _parity(seed, sweep, v):
    # the half-sweep a vertex updates in (label-propagation reading):
    # the low bit of splitmix64(seed ^ splitmix64((sweep << 32) | v)), with
    # splitmix64 pinned to its published output above
    return oracle.splitmix64(seed ^ oracle.splitmix64((sweep << 32) | v)) & 1


def _seed_with_parities(pattern):
    for seed in range(1 << 16):
        if [_parity(seed, 0, v) for v in range(len(pattern))] == pattern:
            return seed
    raise AssertionError("no seed with that parity pattern")


def test_label_prop_half_sweeps_are_synchronous():
    # Unit path 0 - 1 - 2 - 3 - 4, one sweep, every vertex in half-sweep 0.
    # Each vertex takes its neighbours' heaviest label, ties to the smallest,
    # from the labels as they stood before the half-sweep:
    #   v0: {1} -> 1;  v1: {0, 2} tie -> 0;  v2: {1, 3} -> 1;
    #   v3: {2, 4} -> 2;  v4: {3} -> 3;  half-sweep 1 moves no vertex.
    # Result 1, 0, 1, 2, 3.  Updating in place in vertex order would give
    # 1, 1, 1, 1, 1 instead (v1 would already see label 1 at v0, and so on).
    g = graphgen.from_edges(5, np.array([0, 1, 2, 3]), np.array([1, 2, 3, 4]))
    seed = _seed_with_parities([0, 0, 0, 0, 0])
    assert list(oracle.label_prop(*g, iters=1, seed=seed)) == [1, 0, 1, 2, 3]


def test_label_prop_parity_split():
    # The same path with parities 0, 1, 0, 1, 0 in sweep 0.
    # Half-sweep 0 (v0, v2, v4 at once, from 0, 1, 2, 3, 4):
    #   v0 -> 1;  v2: {1, 3} -> 1;  v4 -> 3           labels 1, 1, 1, 3, 3
    # Half-sweep 1 (v1, v3, from those labels):
    #   v1: {0: 1, 2: 1} -> 1 (weight 2);  v3: {2: 1, 4: 3} tie -> 1
    # Result 1, 1, 1, 1, 3.  Without the split (all vertices in both
    # half-sweeps) it would be 0, 1, 0, 1, 2.
    g = graphgen.from_edges(5, np.array([0, 1, 2, 3]), np.array([1, 2, 3, 4]))
    seed = _seed_with_parities([0, 1, 0, 1, 0])
    assert list(oracle.label_prop(*g, iters=1, seed=seed)) == [1, 1, 1, 1, 3]


def test_label_prop_weighted_choice():
    # A star centre 0 with leaves 1 (weight 1), 2 (weight 1), 3 (weight 2)
    # and the edge 2 - 3 (weight 1); every vertex in half-sweep 0.
    # v0: labels 1 (1), 2 (1), 3 (2) -> 3;  v1: {0} -> 0;
    # v2: {0: 1, 3: 1} tie -> 0;  v3: {0: 2, 2: 1} -> 0.
    # Result 3, 0, 0, 0: the heavier arc wins over the smaller label.
    g = graphgen.from_edges(4, np.array([0, 0, 0, 2]), np.array([1, 2, 3, 3]),
                            np.array([1, 1, 2, 1]))
    seed = _seed_with_parities([0, 0, 0, 0])
    assert list(oracle.label_prop(*g, iters=1, seed=seed)) == [3, 0, 0, 0]


def test_planted_4096_two_exact_algorithms_agree():
    # the small plain-method workload: Stoer-Wagner and NOI agree, lambda <= 8
    g = graphgen.planted(1)
    sw, s1 = oracle.stoer_wagner(*g)
    noi, s2, _ = oracle.noi(*g)
    assert sw == noi <= 8
    assert oracle.cut_weight(*g, s1) == sw and oracle.cut_weight(*g, s2) == sw


def _subdivided(rng, i):
    # a small random base graph whose edges are replaced by paths of equal
    # weight (degree-2 chains), plus a few chords
    nb = int(rng.integers(2, 6))
    base = [(a, b) for a in range(nb) for b in range(a + 1, nb) if rng.random() < 0.7]
    if not base:
        base = [(0, 1)]
    u, v, w = [], [], []
    nxt = nb
    for a, b in base:
        k = int(rng.integers(0, 4))
        c = int(rng.integers(1, 4))
        chain = [a] + list(range(nxt, nxt + k)) + [b]
        nxt += k
        for x, y in zip(chain, chain[1:]):
            u.append(x); v.append(y); w.append(c)
    n = nxt
    if n > 16:
        return None
    for _ in range(int(rng.integers(0, 3))):
        x, y = rng.integers(0, n, size=2)
        if x != y:
            u.append(int(x)); v.append(int(y)); w.append(int(rng.integers(1, 4)))
    return n, graphgen.from_edges(n, np.array(u), np.array(v), np.array(w))


def test_pr_degree2_tie_rule_preserves_lambda():
    # the degree-2 tie rule (level >= 2) on graphs full of equal-weight chains
    rng = np.random.default_rng(21)
    checked = 0
    while checked < 400:
        r = _subdivided(rng, checked)
        if r is None:
            continue
        n, g = r
        lam = oracle.brute_force(*g)[0]
        bound = int(oracle.degrees(*g).min())
        lab = oracle.pr_tests(*g, bound, 2)
        roots, lab2 = np.unique(lab, return_inverse=True)
        if len(roots) > 1:
            crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
            lam_c = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))[0]
        else:
            lam_c = bound
        assert min(bound, lam_c) == lam, (checked, bound, lam_c, lam)
        checked += 1


def test_pr_degree2_tie_rule_cycle_and_chain():
    # a unit cycle collapses in one application (lambda = delta = 2) ...
    g = graphgen.cycle(12)
    assert len(np.unique(oracle.pr_tests(*g, 2, 2))) == 1
    # ... and a unit chain between two cliques keeps one chain edge open
    a = 8
    iu, ju = np.triu_indices(a, 1)
    k = 5
    chain = [0] + list(range(2 * a, 2 * a + k)) + [a]
    u = np.concatenate([iu, iu + a, chain[:-1]])
    v = np.concatenate([ju, ju + a, chain[1:]])
    g = graphgen.from_edges(2 * a + k, u, v)
    lab = oracle.pr_tests(*g, 2, 2)
    assert lab[0] != lab[a]
    roots, lab2 = np.unique(lab, return_inverse=True)
    crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
    assert oracle.stoer_wagner(crp.astype(np.int32), ccol, cw.astype(np.int32))[0] == 1


def test_gnn_reference_gradient_matches_finite_differences():
    # the FP64 reference network's analytic backward pass against central
    # differences of its own loss, on small random graphs
    from oracle import gnn
    rng = np.random.default_rng(17)
    for t in range(3):
        g = graphgen.random_connected(30 + 10 * t, 60, seed=200 + t, wmax=9)
        n = len(g[0]) - 1
        side = (rng.random(n) < 0.3).astype(np.int64)
        params = gnn.glorot(t)
        loss, grad = gnn.loss_and_grad(params, *g, side)
        assert abs(loss - gnn.loss_only(params, *g, side)) < 1e-12
        idx = np.concatenate([rng.choice(gnn.P_TOTAL, 40, replace=False),
                              [gnn.P_BOUT, gnn.P_BIN, gnn.P_W0 + 5, gnn.P_W0 + 64 * 64 + 3]])
        num = gnn.numeric_grad(params, *g, side, idx)
        assert np.allclose(grad[idx], num, rtol=1e-4, atol=1e-8), (t, np.max(np.abs(grad[idx] - num)))


def test_gnn_reference_polarity_invariant():
    from oracle import gnn
    g = graphgen.random_connected(25, 50, seed=9, wmax=5)
    n = len(g[0]) - 1
    side = (np.arange(n) % 3 == 0).astype(np.int64)
    p = gnn.glorot(4)
    assert gnn.loss_only(p, *g, side) == gnn.loss_only(p, *g, 1 - side)


def test_gnn_bf16_rounding_matches_torch():
    # the reference's BF16 rounding (nearest, ties to even) against torch's
    # CPU conversion, on hand-picked ties and random values
    import torch
    from oracle import gnn
    ties = np.array([1.0, 1 + 2**-8, 1 + 3 * 2**-8, -(1 + 2**-8), 3.0e-39, 65504.0, 1e30, -2.5e-3])
    assert list(gnn.bf16(ties[:3])) == [1.0, 1.0, 1 + 2**-6]
    x = np.concatenate([ties, np.random.default_rng(3).standard_normal(2000) * 10.0])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert (gnn.bf16(x) == ref).all()


def test_gnn_smoothed_features_separate_two_cliques():
    # two K_20 joined by one edge: the lazy walk evens out each clique long
    # before the two drift together, so after centring the smoothed random
    # features have one sign on each clique (the sparse cut's two sides);
    # they are centred by degree and scaled to magnitude 1
    from oracle import gnn
    iu, ju = np.triu_indices(20, 1)
    g = graphgen.from_edges(40, np.concatenate([iu, iu + 20, [3]]),
                            np.concatenate([ju, ju + 20, [25]]))
    X, G = gnn.features(*g)
    d = G[5]
    for j in (6, 7):
        q = X[:, j]
        assert abs(d @ q) < 1e-9 * d.sum() and np.isclose(np.abs(q).max(), 1.0)
        assert np.sign(q[:20]).min() == np.sign(q[:20]).max() != 0
        assert np.sign(q[20:]).min() == np.sign(q[20:]).max() == -np.sign(q[0])


def test_gnn_bf16_network_close_to_exact():
    # the rounded network stays within BF16 precision of the exact one
    from oracle import gnn
    g = graphgen.random_connected(60, 200, seed=5, wmax=9)
    p = gnn.glorot(8)
    s0, _ = gnn.forward(p, *g)
    s1, _ = gnn.forward(p, *g, bf16_round=True)
    assert 0 < np.linalg.norm(s1 - s0) / np.linalg.norm(s0) < 3e-2


# ---------------------------------------------------- Matula approximation
@pytest.mark.parametrize("a", [500, 400, 250, 1])
def test_matula_guarantee_vs_brute_force(a):
    # Sec. 3.1.1: marking at (1/2 - eps) * delta returns a real cut within
    # a factor 1 / (1/2 - eps) = 1000 / a of lambda
    rng = np.random.default_rng(777 + a)
    loose = 0
    for i in range(800):
        n, g = _random_tiny(rng, i)
        bf, _ = oracle.brute_force(*g)
        cut, side, _ = oracle.matula(*g, a, seed=i)
        assert bf <= cut and cut * a <= bf * 1000, (i, bf, cut, a)
        assert side_ok(side, n) and oracle.cut_weight(*g, side) == cut
        loose += cut > bf
    if a <= 250:
        assert loose > 0  # the threshold really is lower than lambda-hat


def test_matula_exact_where_lambda_is_delta():
    # the answer never exceeds delta, so it is exact whenever lambda = delta
    for n, wt in [(2, 3), (7, 1), (30, 2)]:
        for a in (500, 100):
            assert oracle.matula(*graphgen.complete(n, wt), a)[0] == (n - 1) * wt
            if n >= 3:
                assert oracle.matula(*graphgen.cycle(n, wt), a)[0] == 2 * wt
    g = graphgen.rhg(1, 1 << 12, 16.0)
    lam = oracle.noi(*g)[0]
    if lam == int(oracle.degrees(*g).min()):
        assert oracle.matula(*g, 450)[0] == lam


def test_matula_rejects_bad_settings():
    g = graphgen.cycle(5)
    for a in (0, 501, -3):
        with pytest.raises(Exception):
            oracle.matula(*g, a)


# ------------------------------------------------- one CAPFOREST round
def test_capforest_round_safe_and_progresses():
    # Lemma 1 / Lemma 2: the unions of one capped scan keep
    # min(lambda-hat, lambda(G/U)) = lambda(G); with lambda-hat <= delta and
    # lambda-hat unchanged by the scan, at least one edge is marked (Sec. 2.2)
    rng = np.random.default_rng(4242)
    for i in range(1500):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        lam, _ = oracle.brute_force(*g)
        delta = int(oracle.degrees(*g).min())
        for bound in {delta, lam}:
            if bound <= 0:
                continue
            out, lab = oracle.capforest_round(*g, bound, i % n)
            assert lam <= out <= bound
            roots, lab2 = np.unique(lab, return_inverse=True)
            assert (lab[roots] == roots).all() and (lab <= np.arange(n)).all()
            if len(roots) >= 2:
                crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
                lam_c, _ = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))
                assert min(out, lam_c) == lam, (i, bound, out, lam_c, lam)
            else:
                assert out == lam
            if out == bound and lam > 0:
                assert len(roots) < n


def _noi_by_rounds(g, seed):
    # orc_noi's loop rebuilt from single rounds: the same starts, the same
    # contraction (blocks numbered by their smallest member), the same bound
    cur = g
    lam = int(oracle.degrees(*g).min())
    rounds = 0
    while len(cur[0]) - 1 >= 2 and lam > 0:
        n = len(cur[0]) - 1
        before = lam
        start = oracle.splitmix64(seed ^ rounds) % n
        lam, lab = oracle.capforest_round(*cur, lam, start)
        rounds += 1
        if lam == 0:
            break
        roots, lab2 = np.unique(lab, return_inverse=True)
        if len(roots) == n:
            assert lam < before
            continue
        crp, ccol, cw = oracle.contract(*cur, lab2.astype(np.int32), len(roots))
        cur = (crp.astype(np.int32), ccol, cw.astype(np.int32))
        if len(roots) >= 2:
            lam = min(lam, int(oracle.degrees(*cur).min()))
    return lam, rounds


def test_capforest_rounds_compose_to_noi():
    rng = np.random.default_rng(99)
    for i in range(400):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        lam, _, rounds = oracle.noi(*g, seed=i)
        assert _noi_by_rounds(g, i) == (lam, rounds), i
    g = graphgen.planted(2, block_n=200, avg_deg=10, cross=3)
    lam, _, rounds = oracle.noi(*g, seed=7)
    assert _noi_by_rounds(g, 7) == (lam, rounds)
