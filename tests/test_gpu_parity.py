"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work is compared bit-exact: canonical CSR, degrees, contraction,
Padberg-Rinaldi blocks, and lambda.  A minimum cut's side is not unique, so
the side is checked for validity: proper, canonical polarity, and its
recomputed weight equals lambda.  Concurrent CAPFOREST unions are racy by
design (Sec. 3.2), so a round of them is checked by what the paper's Lemma 2
guarantees: contracting its blocks keeps min(lambda-hat, lambda(G/U)) =
lambda(G).
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


def check_cut(mc, g, res, lam_ref):
    n = len(g[0]) - 1
    side = res.side(n)
    assert res.lam == lam_ref
    assert side[0] == 0
    if lam_ref > 0 or n > 1:
        assert 0 < side.sum() < n
    assert oracle.cut_weight(*g, side) == lam_ref


def assert_root_labels(lab):
    # union-find labels are roots: each points at the smallest vertex of its
    # block, which points at itself
    lab = np.asarray(lab)
    assert (lab[lab] == lab).all() and (lab <= np.arange(len(lab))).all()


def _random_tiny(rng, i):
    n = int(rng.integers(2, 15))
    kind = i % 4
    if kind == 0:
        g = graphgen.random_gnp(n, float(rng.uniform(0.2, 0.9)), seed=i, wmax=100)
    elif kind == 1:
        g = graphgen.random_gnp(n, float(rng.uniform(0.4, 1.0)), seed=i, wmax=3)
    elif kind == 2:
        g = graphgen.random_connected(n, int(rng.integers(0, 3 * n)), seed=i, wmax=10)
    else:
        m = int(rng.integers(1, 3 * n))
        g = graphgen.from_edges(n, rng.integers(0, n, size=m), rng.integers(0, n, size=m),
                                rng.integers(0, 6, size=m))
    return n, g


# ------------------------------------------------------------------ steps --
def test_canonical_export_and_degrees(mc):
    rng = np.random.default_rng(1)
    for i in range(40):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        with mc.Graph(*g) as G:
            rp, col, w = G.export()
            orp, ocol, ow = oracle.contract(*g, np.arange(n, dtype=np.int32), n)
            assert (rp == orp).all() and (col == ocol).all() and (w == ow).all()
            assert (G.degrees() == oracle.degrees(*g)).all()


def test_contract_parity_random_labels(mc):
    rng = np.random.default_rng(2)
    for i in range(30):
        g = graphgen.random_connected(int(rng.integers(20, 3000)), int(rng.integers(0, 20000)),
                                      seed=i, wmax=50)
        n = len(g[0]) - 1
        nc = int(rng.integers(1, n + 1))
        lab = rng.integers(0, nc, size=n).astype(np.int32)
        lab[rng.permutation(n)[:nc]] = np.arange(nc)
        with mc.Graph(*g) as G:
            rp, col, w = G.contract(lab, nc)
        orp, ocol, ow = oracle.contract(*g, lab, nc)
        assert (rp == orp).all() and (col == ocol).all() and (w == ow).all()


def test_contract_clamp(mc):
    g = graphgen.random_connected(500, 4000, seed=5, wmax=50)
    n = len(g[0]) - 1
    lab = (np.arange(n) // 7).astype(np.int32)
    nc = int(lab.max()) + 1
    with mc.Graph(*g) as G:
        rp, col, w = G.contract(lab, nc, clamp=60)
    orp, ocol, ow = oracle.contract(*g, lab, nc)
    assert (rp == orp).all() and (col == ocol).all()
    assert (w == np.minimum(ow, 60)).all()


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_pr_parity(mc, level):
    rng = np.random.default_rng(10 + level)
    for i in range(25):
        g = graphgen.random_connected(int(rng.integers(5, 400)), int(rng.integers(0, 2000)),
                                      seed=100 * level + i, wmax=int(rng.integers(1, 30)))
        deg = oracle.degrees(*g)
        lam = int(deg.min()) - int(rng.integers(0, 3))
        with mc.Graph(*g) as G:
            lab = G.pr_tests(lam, level)
        assert_root_labels(lab)
        assert (lab == oracle.pr_tests(*g, lam, level)).all()


def test_capforest_round_is_safe(mc):
    # Lemma 2: every union of a concurrent capped round keeps the minimum cut
    rng = np.random.default_rng(3)
    for i in range(150):
        n, g = _random_tiny(rng, i)
        if n < 3:
            continue
        lam_g = oracle.brute_force(*g)[0]
        deg = oracle.degrees(*g)
        for budget in (0, 6):
            with mc.Graph(*g) as G:
                lab, lam_out, unions = G.capforest_round(int(deg.min()),
                                                         mc.options(region_budget=budget, seed=i))
            assert_root_labels(lab)
            assert lam_out >= lam_g
            roots, lab2 = np.unique(lab, return_inverse=True)
            if len(roots) == 1:
                assert lam_out == lam_g
                continue
            crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
            lam_c = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))[0] \
                if len(roots) >= 2 else lam_out
            assert min(lam_out, lam_c) == lam_g, (i, lam_out, lam_c, lam_g)


def test_capforest_round_medium_safe(mc):
    for i in range(6):
        g = graphgen.planted(40 + i, block_n=150, avg_deg=10, cross=3)
        lam_g = oracle.stoer_wagner(*g)[0]
        deg = oracle.degrees(*g)
        with mc.Graph(*g) as G:
            lab, lam_out, unions = G.capforest_round(int(deg.min()))
        assert_root_labels(lab)
        assert unions > 0
        roots, lab2 = np.unique(lab, return_inverse=True)
        if len(roots) == 1:
            assert lam_out == lam_g
            continue
        crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
        lam_c = oracle.stoer_wagner(crp.astype(np.int32), ccol, cw.astype(np.int32))[0]
        assert min(lam_out, lam_c) == lam_g


@pytest.mark.parametrize("seed,logn,deg,unites", [(2, 14, 16.0, True), (5, 16, 32.0, True),
                                                  (3, 13, 64.0, True), (6, 12, 90.0, False)])
def test_capforest_round_rhg_safe(mc, seed, logn, deg, unites):
    # thousands of concurrent scans on one graph, lambda-hat 3, 8, 29 and 42
    # (each bitmap queue size): the round keeps min(lambda-hat, lambda(G/U))
    # = lambda(G); at lambda-hat 42 (average degree 90) scans of 48-64
    # vertices reach no threshold, which leaves the work to the full scan
    g = graphgen.rhg(seed, 1 << logn, deg)
    lam_g = oracle.noi(*g)[0]
    d = oracle.degrees(*g)
    for budget in (0, 48):
        with mc.Graph(*g) as G:
            lab, lam_out, unions = G.capforest_round(int(d.min()), mc.options(region_budget=budget, seed=seed))
        assert_root_labels(lab)
        assert lam_out >= lam_g and (unions > 0 or not unites)
        roots, lab2 = np.unique(lab, return_inverse=True)
        if len(roots) == 1:
            assert lam_out == lam_g
            continue
        crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
        lam_c = oracle.noi(crp.astype(np.int32), ccol, cw.astype(np.int32))[0] if len(roots) >= 2 else lam_out
        assert min(lam_out, lam_c) == lam_g


@pytest.mark.parametrize("visits", [2, 3, 8])
def test_capforest_round_with_revisits_safe(mc, visits):
    # Sec. 3.2's variant where a vertex may be scanned by several scans: each
    # scan is still a capped CAPFOREST scan of its own, so a round keeps
    # min(lambda-hat, lambda(G/U)) = lambda(G) (Lemma 2), on tiny graphs
    # (brute force) and on RHG graphs with thousands of concurrent scans
    rng = np.random.default_rng(30 + visits)
    cases = [(oracle.brute_force, _random_tiny(rng, i)[1]) for i in range(120)]
    cases += [(lambda *g: oracle.noi(*g)[:2], graphgen.rhg(s, 1 << 14, 16.0)) for s in (2, 3)]
    for exact, g in cases:
        n = len(g[0]) - 1
        if n < 3:
            continue
        lam_g = exact(*g)[0]
        deg = oracle.degrees(*g)
        for budget in (0, 6):
            with mc.Graph(*g) as G:
                lab, lam_out, unions = G.capforest_round(
                    int(deg.min()), mc.options(region_budget=budget, seed=n, visits=visits))
            assert_root_labels(lab)
            assert lam_out >= lam_g
            roots, lab2 = np.unique(lab, return_inverse=True)
            if len(roots) == 1:
                assert lam_out == lam_g
                continue
            crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
            cg = (crp.astype(np.int32), ccol, cw.astype(np.int32))
            lam_c = oracle.brute_force(*cg)[0] if len(roots) <= 20 else oracle.noi(*cg)[0]
            assert min(lam_out, lam_c) == lam_g, (n, lam_out, lam_c, lam_g)


@pytest.mark.parametrize("visits", [2, 4])
def test_min_cut_with_revisits(mc, visits):
    # lambda and its side with several scans per vertex, on the plain-path
    # workload shapes (planted blocks, RHG, an R-MAT k-core)
    for g in (graphgen.planted(1), graphgen.rhg(3, 1 << 17, 32.0), graphgen.rmat_kcore(2, scale=17, k=10),
              graphgen.planted_rhg(3, 1 << 15, 32.0, cross=3)):
        ref, _, _ = oracle.noi(*g)
        with mc.Graph(*g) as G:
            res = G.min_cut(mc.options(visits=visits))
        check_cut(mc, g, res, ref)


# ------------------------------------------------------------ full solves --
def test_random_tiny_min_cut(mc):
    rng = np.random.default_rng(4)
    for i in range(400):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        ref = oracle.brute_force(*g)[0]
        with mc.Graph(*g) as G:
            # a third of the cases skip the single-warp tail solver
            res = G.min_cut(mc.options(seed=i, pq_order=i % 2, pr_level=i % 5,
                                       tail_vertices=-1 if i % 3 == 0 else 0))
        check_cut(mc, g, res, ref)


@pytest.mark.parametrize("n,wt", [(2, 1), (3, 4), (10, 1), (33, 3), (100, 1)])
def test_closed_form_complete(mc, n, wt):
    g = graphgen.complete(n, wt)
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, (n - 1) * wt)


@pytest.mark.parametrize("n,wt", [(3, 1), (50, 7), (5000, 2)])
def test_closed_form_cycle(mc, n, wt):
    g = graphgen.cycle(n, wt)
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, 2 * wt)


def test_closed_form_two_cliques(mc):
    for a, k in [(10, 3), (40, 7), (200, 11)]:
        g = graphgen.two_cliques(a, k, seed=a)
        with mc.Graph(*g) as G:
            res = G.min_cut()
        check_cut(mc, g, res, k)


def test_disconnected_graph(mc):
    g = graphgen.from_edges(7, np.array([0, 1, 3, 4, 5]), np.array([1, 2, 4, 5, 6]),
                            np.array([3, 4, 5, 6, 7]))
    with mc.Graph(*g) as G:
        res = G.min_cut()
    side = res.side(7)
    assert res.lam == 0 and oracle.cut_weight(*g, side) == 0 and side[0] == 0 and side.sum() == 4


def _disjoint_union(parts):
    rps, cols, ws, off, base = [np.zeros(1, np.int64)], [], [], 0, 0
    for rp, col, w in parts:
        rps.append(rp[1:].astype(np.int64) + base)
        cols.append(col.astype(np.int64) + off)
        ws.append(w)
        off += len(rp) - 1
        base += len(col)
    return (np.concatenate(rps).astype(np.int32), np.concatenate(cols).astype(np.int32),
            np.concatenate(ws).astype(np.int32))


@pytest.mark.parametrize("opts", [dict(), dict(tail_vertices=-1), dict(bound=1), dict(pr_level=0)])
def test_disconnected_components_side(mc, opts):
    # lambda = 0 is reached by the exact loop itself; the side is every
    # component but vertex 0's
    parts = [graphgen.random_connected(300, 900, seed=1, wmax=5), graphgen.random_connected(500, 2000, seed=2),
             graphgen.random_connected(50, 100, seed=3, wmax=9), graphgen.complete(40, 3)]
    g = _disjoint_union(parts)
    sizes = [len(p[0]) - 1 for p in parts]
    with mc.Graph(*g) as G:
        res = G.min_cut(mc.options(**opts))
    side = res.side(len(g[0]) - 1)
    assert res.lam == 0 and oracle.cut_weight(*g, side) == 0
    assert (side[:sizes[0]] == 0).all() and (side[sizes[0]:] == 1).all()
    # an isolated vertex: delta = 0 from the start
    g2 = _disjoint_union([parts[0], (np.zeros(2, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))])
    with mc.Graph(*g2) as G:
        res = G.min_cut(mc.options(**opts))
    side = res.side(len(g2[0]) - 1)
    assert res.lam == 0 and side.sum() == 1 and side[-1] == 1


@pytest.mark.parametrize("hub_w", [1, 2, 7])
def test_hub_rows_passed_over(mc, hub_w):
    # a wheel whose hub row (6000 arcs) is longer than the concurrent scans
    # take: the hub is never scanned by them, only touched and united
    k = 6000
    rim = np.arange(k)
    src = np.concatenate([rim, rim])
    dst = np.concatenate([(rim + 1) % k, np.full(k, k)])
    wt = np.concatenate([np.full(k, 3), np.full(k, hub_w)])
    g = graphgen.from_edges(k + 1, src, dst, wt)
    ref = oracle.noi(*g)[0]
    assert ref == min(6 + hub_w, 2 * 3 + 2 * hub_w, k * hub_w)
    for tail in (0, -1):
        with mc.Graph(*g) as G:
            res = G.min_cut(mc.options(tail_vertices=tail))
        check_cut(mc, g, res, ref)


def test_weight_limits(mc):
    big = 2**31 - 4
    # the largest minimum degree the int32 scans accept (2^31 - 3 and up are
    # refused)
    g = graphgen.from_edges(3, np.array([0, 1]), np.array([1, 2]), np.array([big, big]))
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, big)
    g = graphgen.from_edges(3, np.array([0, 1]), np.array([1, 2]), np.array([big + 1, big + 1]))
    with mc.Graph(*g) as G:
        with pytest.raises(mc.MinCutError) as e:
            G.min_cut()
    assert e.value.code == mc.MC_EOVERFLOW
    # parallel arcs summing past INT32_MAX are refused when merged
    g = graphgen.from_edges(2, np.array([0, 0, 0]), np.array([1, 1, 1]), np.array([2**30] * 3))
    with pytest.raises(mc.MinCutError) as e:
        mc.Graph(*g)
    assert e.value.code == mc.MC_EOVERFLOW
    # a minimum degree past the scans' int32 range
    g = graphgen.complete(4, 2**30)
    with mc.Graph(*g) as G:
        with pytest.raises(mc.MinCutError) as e:
            G.min_cut()
    assert e.value.code == mc.MC_EOVERFLOW


def test_tree_and_path(mc):
    for seed in range(5):
        g = graphgen.random_tree(3000, seed)
        with mc.Graph(*g) as G:
            res = G.min_cut()
        check_cut(mc, g, res, int(g[2].min()))


def test_medium_random_vs_stoer_wagner(mc):
    for i in range(10):
        g = graphgen.random_connected(200 + 150 * i, 600 + 900 * i, seed=1000 + i,
                                      wmax=[1, 5, 100][i % 3])
        ref = oracle.stoer_wagner(*g)[0]
        for seed in range(2):
            with mc.Graph(*g) as G:
                res = G.min_cut(mc.options(seed=seed, pq_order=seed))
            check_cut(mc, g, res, ref)


@pytest.mark.parametrize("tail", [-1, 64, 1024, 4096])
def test_tail_solver_sizes(mc, tail):
    # the single-warp tail takes over at different sizes (4096: from the
    # start, with its r-values in global memory past 2048 vertices)
    cases = [graphgen.random_connected(300 + 400 * i, 900 + 1500 * i, seed=70 + i, wmax=[1, 9, 60][i % 3])
             for i in range(5)] + [graphgen.two_cliques(300, 5, seed=3), graphgen.planted(0)]
    for i, g in enumerate(cases):
        ref = oracle.stoer_wagner(*g)[0] if len(g[0]) <= 2000 else oracle.noi(*g)[0]
        with mc.Graph(*g) as G:
            res = G.min_cut(mc.options(seed=i, tail_vertices=tail))
        check_cut(mc, g, res, ref)
        n, arcs = len(g[0]) - 1, len(g[1])
        if tail == 4096 and n <= 4096 and arcs <= 64 * 4096:
            assert res.stats["tail_launches"] == 1 and res.stats["rounds"] == 0
        if tail == -1:
            assert res.stats["tail_launches"] == 0


def test_tail_option_checks(mc):
    g = graphgen.cycle(10, 3)
    with mc.Graph(*g) as G:
        for bad in (-1, 501):
            with pytest.raises(mc.MinCutError):
                G.min_cut(mc.options(approx_milli=bad))
        assert G.min_cut(mc.options(tail_vertices=1 << 20)).lam == 6


def _approx_ok(mc, g, res, lam, a):
    # Matula's guarantee: a real cut, at most 1000 / a times lambda
    n = len(g[0]) - 1
    assert lam <= res.lam and res.lam * a <= lam * 1000, (lam, res.lam, a)
    side = res.side(n)
    assert side[0] == 0 and 0 < side.sum() < n
    assert oracle.cut_weight(*g, side) == res.lam


def test_approx_mode_tiny(mc):
    rng = np.random.default_rng(21)
    for i in range(300):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        lam = oracle.brute_force(*g)[0]
        with mc.Graph(*g) as G:
            for a in (500, 400, 250, 1):
                _approx_ok(mc, g, G.min_cut(mc.options(approx_milli=a, seed=i)), lam, a)


@pytest.mark.parametrize("a", [500, 450, 300])
def test_approx_mode_workloads(mc, a):
    # planted (lambda = 8 below delta), RHG (lambda = delta), a weighted
    # R-MAT core, the LP bound in front, and a disconnected graph (0)
    cases = [(graphgen.planted(1), {}), (graphgen.rhg(2, 1 << 16, 32.0), {}),
             (graphgen.rmat_kcore(1, scale=15), {}), (graphgen.rhg(4, 1 << 15, 32.0), {"bound": 1})]
    for g, kw in cases:
        lam = oracle.noi(*g)[0]
        with mc.Graph(*g) as G:
            exact = G.min_cut(mc.options(**kw)).lam
            res = G.min_cut(mc.options(approx_milli=a, **kw))
        assert exact == lam
        _approx_ok(mc, g, res, lam, a)
    g = graphgen.from_edges(6, np.array([0, 1, 3, 4]), np.array([1, 2, 4, 5]), np.array([5, 5, 5, 5]))
    with mc.Graph(*g) as G:
        assert G.min_cut(mc.options(approx_milli=a)).lam == 0


@pytest.mark.parametrize("seed", range(10))
def test_planted_4096(mc, seed):
    # the small plain-method workload, all ten seeds
    g = graphgen.planted(seed)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, ref)


def test_options_do_not_change_lambda(mc):
    g = graphgen.rhg(5, 1 << 14, 24.0)
    ref, _, _ = oracle.noi(*g)
    for o in [dict(), dict(pq_order=1), dict(pr_level=0), dict(pr_level=4),
              dict(region_budget=64), dict(region_budget=1500), dict(scans_per_round=64),
              dict(seed=99)]:
        with mc.Graph(*g) as G:
            res = G.min_cut(mc.options(**o))
        check_cut(mc, g, res, ref)


def test_device_pointer_graph(mc):
    import torch
    g = graphgen.planted(3, block_n=300, avg_deg=12, cross=4)
    ref, _, _ = oracle.noi(*g)
    t = [torch.from_numpy(a.copy()).cuda() for a in g]
    with mc.Graph(*t) as G:
        res = G.min_cut()
    assert res.lam == ref
    side = res.side(len(g[0]) - 1)
    assert oracle.cut_weight(*g, side) == ref


def test_unweighted_input(mc):
    # w = NULL: every arc has weight 1, on both the one-pass build (canonical
    # rows) and the sort path (parallel arcs become weight 2, self-loops drop)
    import torch
    rng = np.random.default_rng(7)
    for i in range(24):
        n = int(rng.integers(2, 40))
        m = int(rng.integers(1, 4 * n))
        u, v = rng.integers(0, n, size=m), rng.integers(0, n, size=m)
        if i % 2 == 0:  # canonical: distinct edges, no self-loops
            e = np.unique(np.stack([np.minimum(u, v), np.maximum(u, v)], 1)[u != v], axis=0)
            u, v = e[:, 0], e[:, 1]
        # odd i: the raw edge list with its parallel edges and self-loops
        g = graphgen.from_edges(n, u, v)
        ones = (g[0], g[1], np.ones_like(g[2]))
        orp, ocol, ow = oracle.contract(*ones, np.arange(n, dtype=np.int32), n)
        ref = oracle.brute_force(*ones)[0] if n <= 16 else oracle.noi(*ones)[0]
        for dev in (False, True):
            args = [torch.from_numpy(a.copy()).cuda() for a in ones[:2]] if dev else list(ones[:2])
            with mc.Graph(*args) as G:
                rp, col, w = G.export()
                assert (rp == orp).all() and (col == ocol).all() and (w == ow).all()
                res = G.min_cut()
            assert res.lam == ref
            assert oracle.cut_weight(*ones, res.side(n)) == ref
    g = graphgen.rhg(3, 1 << 14, 16.0)
    assert (g[2] == 1).all()
    with mc.Graph(g[0], g[1]) as G:
        assert G.min_cut().lam == oracle.noi(*g)[0]
    # the symmetry check still applies
    bad = (np.array([0, 1, 1], dtype=np.int32), np.array([1], dtype=np.int32))
    with pytest.raises(mc.MinCutError):
        mc.Graph(*bad)


def test_pinned_host_input(mc):
    # page-locked host arrays (the end-to-end benchmark's inputs): the
    # canonical graph, the sort path (parallel arcs, self-loops, unsorted
    # rows, zero weights) and the error checks are the same as from pageable
    # memory
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    rng = np.random.default_rng(11)
    for i in range(16):
        n, g = _random_tiny(rng, i)
        if n < 2:
            continue
        gp = [pin(a) for a in g]
        orp, ocol, ow = oracle.contract(*g, np.arange(n, dtype=np.int32), n)
        with mc.Graph(*gp) as G:
            rp, col, w = G.export()
            assert (rp == orp).all() and (col == ocol).all() and (w == ow).all()
            assert G.min_cut().lam == oracle.brute_force(*g)[0]
    g = graphgen.rhg(2, 1 << 14, 16.0)
    ref = oracle.noi(*g)[0]
    with mc.Graph(pin(g[0]), pin(g[1])) as G:
        assert G.min_cut().lam == ref
    with mc.Graph(*[pin(a) for a in g]) as G:
        assert G.min_cut().lam == ref
    bad = [pin(a) for a in (np.array([0, 1, 1], dtype=np.int32), np.array([1], dtype=np.int32),
                            np.array([1], dtype=np.int32))]
    with pytest.raises(mc.MinCutError):
        mc.Graph(*bad)
    bad[1][0] = 7  # out of range
    with pytest.raises(mc.MinCutError):
        mc.Graph(*bad)


def test_input_conventions(mc):
    # parallel arcs summed, self-loops and zero weights dropped
    g = graphgen.from_edges(4, np.array([0, 0, 1, 2, 3, 1, 2]), np.array([1, 1, 2, 3, 3, 3, 0]),
                            np.array([2, 3, 4, 5, 50, 0, 1]))
    ref = oracle.brute_force(*g)[0]
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, ref)


def test_invalid_inputs(mc):
    rp = np.array([0, 1, 1], dtype=np.int32)  # arc 0->1 without its mirror
    with pytest.raises(mc.MinCutError) as e:
        mc.Graph(rp, np.array([1], dtype=np.int32), np.array([1], dtype=np.int32))
    assert e.value.code == -1
    rp, col, w = graphgen.cycle(5)
    bad = col.copy()
    bad[0] = 9
    with pytest.raises(mc.MinCutError):
        mc.Graph(rp, bad, w)
    neg = w.copy()
    neg[:] = -1
    with pytest.raises(mc.MinCutError):
        mc.Graph(rp, col, neg)
    badrp = rp.copy()
    badrp[2] = 0
    with pytest.raises(mc.MinCutError):
        mc.Graph(badrp, col, w)


def test_asymmetric_graph_rejected(mc):
    # canonical input (sorted rows) is checked on its own arrays, other input
    # on its canonical form; both refuse a missing mirror or a mirror of
    # another weight, with and without a weight array
    g = graphgen.random_connected(300, 900, seed=3, wmax=9)
    rp, col, w = (np.asarray(a, dtype=np.int32) for a in oracle.contract(*g, np.arange(300, dtype=np.int32), 300))
    assert all((np.diff(col[rp[v]:rp[v + 1]]) > 0).all() for v in range(300))  # canonical as given
    with mc.Graph(rp, col, w) as G:
        assert G.min_cut().lam == oracle.noi(rp, col, w)[0]
    w_bad = w.copy()
    w_bad[5] += 1
    rp_d = np.array([0, 1, 2, 3], dtype=np.int32)    # 0 -> 1, 1 -> 0, and 2 -> 0 unmirrored
    col_d = np.array([1, 0, 0], dtype=np.int32)
    for args in ((rp, col, w_bad), (rp_d, col_d, np.ones(3, dtype=np.int32)), (rp_d, col_d, None)):
        with pytest.raises(mc.MinCutError) as e:
            mc.Graph(*args)
        assert e.value.code == mc.MC_EINVAL
    # the same weight mismatch with a reversed row (not canonical as given)
    col_r, w_r = col.copy(), w_bad.copy()
    col_r[rp[0]:rp[1]] = col_r[rp[0]:rp[1]][::-1].copy()
    w_r[rp[0]:rp[1]] = w_r[rp[0]:rp[1]][::-1].copy()
    with pytest.raises(mc.MinCutError) as e:
        mc.Graph(rp, col_r, w_r)
    assert e.value.code == mc.MC_EINVAL


def _check_batch_sides(b, lam, bits, boff, ks):
    for k in ks:
        g = graphgen.batch_graph(b, k)
        n = len(g[0]) - 1
        side = np.unpackbits(bits[boff[k]:boff[k + 1]].view(np.uint8), bitorder="little")[:n]
        assert side[0] == 0 and 0 < side.sum() < n
        assert oracle.cut_weight(*g, side) == lam[k], k


def test_batch_small(mc):
    b = graphgen.batch(7, G=48)
    lam, bits, boff, st = mc.batch_min_cut(*b, bitmaps=True)
    for k in range(48):
        g = graphgen.batch_graph(b, k)
        assert lam[k] == oracle.noi(*g)[0], k
    _check_batch_sides(b, lam, bits, boff, range(48))


def test_batch_sharded_ranges(mc):
    # the per-rank ranges of a sharded batch, each solved by its own
    # mc_batch_min_cut call, give the whole batch's lambdas
    from paper_1808_05458_gb300 import shard
    b = graphgen.batch(8, G=40)
    full = mc.batch_min_cut(*b)[0]
    for world in (1, 3, 7):
        bounds = shard.shard_bounds(b[3], b[4], world)
        parts = [mc.batch_min_cut(*shard.sub_batch(b, int(bounds[r]), int(bounds[r + 1])))[0]
                 for r in range(world) if bounds[r + 1] > bounds[r]]
        assert (np.concatenate(parts) == full).all()
    lam = shard.sharded_batch_min_cut(b, 0, 1, lambda x: [x])
    assert (lam == full).all()
    assert all(full[k] == oracle.noi(*graphgen.batch_graph(b, k))[0] for k in range(40))


def test_batch_graph_replay(mc):
    # the persistent launch is captured once per batch layout and replayed:
    # repeated calls, then another layout, then the first again
    b1, b2 = graphgen.batch(11, G=64), graphgen.batch(12, G=40)
    ref1 = [oracle.noi(*graphgen.batch_graph(b1, k))[0] for k in range(64)]
    ref2 = [oracle.noi(*graphgen.batch_graph(b2, k))[0] for k in range(40)]
    for b, ref in [(b1, ref1), (b1, ref1), (b1, ref1), (b2, ref2), (b1, ref1)]:
        lam, bits, boff, _ = mc.batch_min_cut(*b, bitmaps=True)
        assert list(lam) == ref
        _check_batch_sides(b, lam, bits, boff, range(len(ref)))


def _concat(graphs):
    rps, cols, ws, voff, aoff = [], [], [], [0], [0]
    for rp, col, w in graphs:
        rps.append(rp)
        cols.append(col)
        ws.append(w)
        voff.append(voff[-1] + len(rp) - 1)
        aoff.append(aoff[-1] + len(col))
    return (np.concatenate(rps).astype(np.int32), np.concatenate(cols).astype(np.int32),
            np.concatenate(ws).astype(np.int32), np.array(voff, dtype=np.int64),
            np.array(aoff, dtype=np.int64))


def test_batch_edge_cases(mc):
    rng = np.random.default_rng(9)
    graphs = [graphgen.from_edges(2, np.array([0]), np.array([1]), np.array([5])),
              graphgen.from_edges(5, np.array([0, 1, 3]), np.array([1, 2, 4]), np.array([3, 3, 3])),
              graphgen.cycle(40, 3), graphgen.complete(20, 2), graphgen.two_cliques(30, 4, seed=2),
              graphgen.from_edges(4, np.array([0, 0, 1, 2, 3, 1]), np.array([1, 1, 2, 3, 3, 3]),
                                  np.array([2, 3, 4, 5, 50, 0]))]
    for i in range(40):
        graphs.append(_random_tiny(rng, 1000 + i)[1])
    graphs = [g for g in graphs if len(g[0]) - 1 >= 2]
    b = _concat(graphs)
    lam, bits, boff, _ = mc.batch_min_cut(*b, bitmaps=True)
    for k, g in enumerate(graphs):
        n = len(g[0]) - 1
        ref = oracle.brute_force(*g)[0] if n <= 16 else oracle.stoer_wagner(*g)[0]
        assert lam[k] == ref, (k, lam[k], ref)
        side = np.unpackbits(bits[boff[k]:boff[k + 1]].view(np.uint8), bitorder="little")[:n]
        assert side[0] == 0 and 0 < side.sum() < n and oracle.cut_weight(*g, side) == ref


def test_batch_invalid(mc):
    rp, col, w = graphgen.cycle(6)
    bad = col.copy()
    bad[3] = 17
    b = _concat([(rp, bad, w)])
    with pytest.raises(mc.MinCutError):
        mc.batch_min_cut(*b)
    b = _concat([(rp, col, -w)])
    with pytest.raises(mc.MinCutError):
        mc.batch_min_cut(*b)
    # a row offset that falls (the ends right): refused before any arc is read
    good = graphgen.complete(5, 2)
    rp_f = rp.copy()
    rp_f[2] = rp_f[1] - 1
    for graphs in ([(rp_f, col, w)], [good, (rp_f, col, w), good]):
        with pytest.raises(mc.MinCutError) as ei:
            mc.batch_min_cut(*_concat(graphs))
        assert ei.value.code == mc.MC_EINVAL


def test_batch_asymmetric_rejected(mc):
    # a graph whose arc lacks its mirror, or whose mirror has another weight,
    # is malformed input: the whole call returns MC_EINVAL
    rp, col, w = graphgen.cycle(7, 3)
    good = graphgen.complete(5, 2)
    w_bad = w.copy()
    w_bad[0] += 1                      # (0, 1, 4) against (1, 0, 3)
    rp_m = np.array([0, 1, 2, 2], dtype=np.int32)   # 0 -> 1 and 1 -> 2 without mirrors
    col_m = np.array([1, 2], dtype=np.int32)
    w_m = np.array([1, 1], dtype=np.int32)
    # every upward arc has its mirror, but the downward arc 2 -> 0 has none
    # (as many arcs down as up fails)
    g_down = (np.array([0, 1, 2, 3], dtype=np.int32), np.array([1, 0, 0], dtype=np.int32),
              np.array([1, 1, 1], dtype=np.int32))
    # a downward arc whose mirror row is empty
    g_empty = (np.array([0, 0, 1], dtype=np.int32), np.array([0], dtype=np.int32), np.array([4], dtype=np.int32))
    for bad in ((rp, col, w_bad), (rp_m, col_m, w_m), g_down, g_empty):
        for graphs in ([bad], [good, bad, good]):
            with pytest.raises(mc.MinCutError) as ei:
                mc.batch_min_cut(*_concat(graphs))
            assert ei.value.code == mc.MC_EINVAL
    # parallel arcs that merge into a symmetric graph are accepted: 0 -> 1
    # given as 2 + 3 in row 0 and as 5 in row 1
    rp_p = np.array([0, 2, 3], dtype=np.int32)
    g_par = (rp_p, np.array([1, 1, 0], dtype=np.int32), np.array([2, 3, 5], dtype=np.int32))
    lam, _, _, _ = mc.batch_min_cut(*_concat([good, g_par]))
    assert list(lam) == [8, 5]
    # rows out of neighbour order take the transpose-based check: a
    # symmetric graph so given is solved, an asymmetric one refused
    def reverse_rows(g):
        rp_, col_, w_ = (np.array(a) for a in g)
        for v in range(len(rp_) - 1):
            col_[rp_[v]:rp_[v + 1]] = col_[rp_[v]:rp_[v + 1]][::-1].copy()
            w_[rp_[v]:rp_[v + 1]] = w_[rp_[v]:rp_[v + 1]][::-1].copy()
        return rp_, col_, w_
    rev = reverse_rows(graphgen.two_cliques(9, 2, seed=4))
    lam, _, _, _ = mc.batch_min_cut(*_concat([rev, good]))
    assert list(lam) == [2, 8]
    with pytest.raises(mc.MinCutError) as ei:
        mc.batch_min_cut(*_concat([reverse_rows((rp, col, w_bad))]))
    assert ei.value.code == mc.MC_EINVAL


def test_batch_4096_full(mc):
    # the batched workload: 4096 graphs, n in 50..2000, degree 4..16, weights 1..100
    b = graphgen.batch(1)
    lam, bits, boff, st = mc.batch_min_cut(*b, bitmaps=True)
    ref = np.array([oracle.noi(*graphgen.batch_graph(b, k))[0] for k in range(4096)])
    assert (lam == ref).all(), np.nonzero(lam != ref)[0][:10]
    _check_batch_sides(b, lam, bits, boff, range(0, 4096, 7))
    # Stoer-Wagner on a sample of the small graphs
    small = [k for k in range(4096) if b[3][k + 1] - b[3][k] <= 150][:24]
    for k in small:
        assert lam[k] == oracle.stoer_wagner(*graphgen.batch_graph(b, k))[0]


def test_batch_every_shape_and_autotune(mc):
    b = graphgen.batch(3, G=256)
    ref, _, _, _ = mc.batch_min_cut(*b)
    best, ms = mc.batch_autotune(*b)
    k = mc.batch_shape_count()
    assert 0 <= best < k and (ms[:k] > 0).all()
    lam, _, _, _ = mc.batch_min_cut(*b)
    assert (lam == ref).all()


def _reverse_rows(g):
    rp, col, w = (np.array(a) for a in g)
    for v in range(len(rp) - 1):
        col[rp[v]:rp[v + 1]] = col[rp[v]:rp[v + 1]][::-1].copy()
        w[rp[v]:rp[v + 1]] = w[rp[v]:rp[v + 1]][::-1].copy()
    return rp, col, w


def test_batch_every_shape_exact_at_size_boundaries(mc):
    # each kernel shape (shared vertices per warp 512, 1024 or 2048) on graphs
    # just below, at and above those sizes and the 16-bit union-find's limit
    # (SN - 2): on-chip and global paths alike; caps of 2^25 and above take
    # the bucket-list scan; reversed rows take the general canonicalisation
    sizes = (2, 3, 33, 65, 254, 255, 256, 257, 510, 511, 512, 513, 1022, 1023, 1024, 1025,
             2046, 2047, 2048, 2049)
    graphs = [graphgen.random_connected(n, 2 * n, seed=300 + i, wmax=100) for i, n in enumerate(sizes)]
    heavy = graphgen.random_connected(300, 600, seed=7, wmax=100)
    graphs.append((heavy[0], heavy[1], ((heavy[2].astype(np.int64) + 128) << 18).astype(np.int32)))
    graphs.append(_reverse_rows(graphgen.random_connected(700, 1400, seed=8, wmax=100)))
    graphs.append(_reverse_rows(graphgen.random_connected(1023, 2000, seed=9, wmax=100)))
    graphs.append(graphgen.two_cliques(40, 3, seed=5))
    b = _concat(graphs)
    ref = [oracle.noi(*g)[0] for g in graphs]
    try:
        for k in range(mc.batch_shape_count()):
            mc.batch_set_shape(k)
            for order in (mc.MC_PQ_LIFO, mc.MC_PQ_FIFO):
                lam, bits, boff, _ = mc.batch_min_cut(*b, mc.options(pq_order=order), bitmaps=True)
                assert list(lam) == ref, (k, order, [(i, lam[i], ref[i]) for i in range(len(ref)) if lam[i] != ref[i]])
                _check_batch_sides(b, lam, bits, boff, range(len(graphs)))
        with pytest.raises(mc.MinCutError):
            mc.batch_set_shape(mc.batch_shape_count())
    finally:
        mc.batch_set_shape(-1)


def test_batch_random_kinds_every_shape(mc):
    # mixed kinds per shape: dense graphs (contracted rows far past 32 arcs),
    # sparse and disconnected ones, raw edge lists with loops, repeats and
    # zero weights, heavy weights, and cliques joined by a few edges
    rng = np.random.default_rng(77)
    graphs = []
    for i in range(120):
        kind = i % 6
        if kind == 0:
            n = int(rng.integers(40, 260))
            g = graphgen.random_gnp(n, float(rng.uniform(0.2, 0.6)), seed=500 + i, wmax=int(rng.integers(1, 50)))
        elif kind == 1:
            n = int(rng.integers(100, 2100))
            g = graphgen.random_connected(n, int(rng.integers(n, 6 * n)), seed=500 + i, wmax=100)
        elif kind == 2:
            n = int(rng.integers(20, 400))
            g = graphgen.random_gnp(n, float(rng.uniform(0.002, 0.02)), seed=500 + i, wmax=10)
        elif kind == 3:
            n = int(rng.integers(10, 900))
            m = int(rng.integers(n, 8 * n))
            g = graphgen.from_edges(n, rng.integers(0, n, size=m), rng.integers(0, n, size=m),
                                    rng.integers(0, 5, size=m))
        elif kind == 4:
            n = int(rng.integers(50, 1500))
            g0 = graphgen.random_connected(n, 3 * n, seed=500 + i, wmax=100)
            g = (g0[0], g0[1], ((g0[2].astype(np.int64) + 128) << 17).astype(np.int32))
        else:
            g = graphgen.two_cliques(int(rng.integers(10, 60)), int(rng.integers(1, 6)), seed=500 + i)
        if len(g[0]) - 1 >= 2:
            graphs.append(g)
    b = _concat(graphs)
    ref = [oracle.noi(*g)[0] for g in graphs]
    try:
        for k in range(mc.batch_shape_count()):
            mc.batch_set_shape(k)
            lam, bits, boff, _ = mc.batch_min_cut(*b, bitmaps=True)
            bad = [(i, lam[i], ref[i]) for i in range(len(ref)) if lam[i] != ref[i]]
            assert not bad, (k, bad[:5])
            _check_batch_sides(b, lam, bits, boff, [i for i in range(len(graphs)) if ref[i] > 0])
    finally:
        mc.batch_set_shape(-1)


# ------------------------------------------------------------ full sizes --
def test_rhg_2_20_full_size(mc):
    # the plain-path workload: RHG n = 2^20, average degree 32, exponent 5
    g = graphgen.rhg(1, 1 << 20, 32.0, 5.0)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, ref)


def test_rmat_kcore_scale20(mc):
    g = graphgen.rmat_kcore(1, scale=20)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        res = G.min_cut()
    check_cut(mc, g, res, ref)


@pytest.mark.parametrize("k,order", [(50, 0), (100, 1)])
def test_rmat_dense_kcores(mc, k, order):
    # deeper k-cores of a Kronecker (R-MAT) graph, as the paper's real-world
    # k-core inputs, in both bucket orders
    g = graphgen.rmat_kcore(2, scale=18, k=k)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        res = G.min_cut(mc.options(pq_order=order))
    check_cut(mc, g, res, ref)


def test_capforest_full_scan_safe_and_progresses(mc):
    # Alg. 3: a full scan at lambda-hat <= delta unites at least one edge
    # unless alpha lowered lambda-hat during the scan (Sec. 2.2), and every
    # union keeps min(lambda-hat, lambda(G/U)) = lambda(G) (Lemma 1)
    rng = np.random.default_rng(8)
    for i in range(200):
        n, g = _random_tiny(rng, i)
        if n < 3:
            continue
        lam_g = oracle.brute_force(*g)[0]
        deg = oracle.degrees(*g)
        bound = int(deg.min())
        if bound == 0:
            continue
        with mc.Graph(*g) as G:
            lab, lam_out, unions = G.capforest_full(bound, start=i % n)
            lab2_again, lam2, un2 = G.capforest_full(bound, start=i % n)
        assert (lab == lab2_again).all() and lam_out == lam2 and unions == un2  # deterministic
        assert_root_labels(lab)
        assert lam_out >= lam_g
        if lam_out == bound and lam_g > 0:
            assert unions >= 1
        roots, lab2 = np.unique(lab, return_inverse=True)
        if len(roots) == 1:
            assert lam_out == lam_g
            continue
        crp, ccol, cw = oracle.contract(*g, lab2.astype(np.int32), len(roots))
        lam_c = oracle.brute_force(crp.astype(np.int32), ccol, cw.astype(np.int32))[0]
        assert min(lam_out, lam_c) == lam_g, (i, lam_out, lam_c, lam_g)


def test_full_scan_deterministic_on_ties(mc):
    # unit weights make many equal keys; the scan order among them (and so
    # the set of unions) must not depend on hardware arbitration
    for g in (graphgen.planted(2), graphgen.rhg(4, 1 << 13, 20.0), graphgen.cycle(300),
              graphgen.rhg(6, 1 << 16, 24.0)):
        with mc.Graph(*g) as G:
            lam = int(G.degrees().min())
            runs = [G.capforest_full(lam, start=5) for _ in range(6)]
        for lab, lo, un in runs:
            assert_root_labels(lab)
        for lab, lo, un in runs[1:]:
            assert (lab == runs[0][0]).all() and lo == runs[0][1] and un == runs[0][2]


def _exact_full_scan_cases():
    rng = np.random.default_rng(31)
    cases = [_random_tiny(rng, i)[1] for i in range(120)]
    cases += [graphgen.random_connected(400, 2500, seed=5, wmax=30),
              graphgen.planted(3),                                  # one-warp scan, n <= 4096
              graphgen.planted(5, block_n=3000, avg_deg=40.0, cross=6),  # n 6000, rows of 3 chunks
              graphgen.random_gnp(200, 0.2, seed=21, wmax=2),       # cap 40, rows of 2 chunks
              graphgen.planted(6, block_n=5000, avg_deg=16.0, cross=4),  # block scan, state on chip
              graphgen.rhg(7, 1 << 15, 24.0),                       # block scan, state off chip
              graphgen.rmat_kcore(3, scale=16, k=24),               # a deep core, cap ~ 50
              graphgen.cycle(2000, 3)]
    return cases


def test_full_scan_exact_parity_with_the_oracle(mc):
    # The full scan takes the largest key, ties to the smallest vertex -- the
    # oracle's order -- so while lambda-hat does not drop inside the scan its
    # unions are the oracle's exactly (Alg. 3): at the bound lambda (no cut
    # can lower it) from several starts, and at the bound delta whenever the
    # scan returns it unchanged.
    checked = 0
    for k, g in enumerate(_exact_full_scan_cases()):
        n = len(g[0]) - 1
        if n < 2:
            continue
        deg = oracle.degrees(*g)
        lam = oracle.noi(*g)[0] if n > 20 else oracle.brute_force(*g)[0]
        with mc.Graph(*g) as G:
            for bound in sorted({lam, int(deg.min())}):
                if bound <= 0:
                    continue
                for start in (0, n // 2, n - 1):
                    lab, lam_out, _ = G.capforest_full(bound, start=start)
                    ref_lam, ref_lab = oracle.capforest_round(*g, bound, start)
                    if lam_out == bound and ref_lam == bound:
                        assert (lab == ref_lab).all(), (k, bound, start)
                        checked += 1
    assert checked > 200


@pytest.mark.parametrize("iters", [1, 3])
def test_label_prop_parity(mc, iters):
    # bit-exact against the oracle's reading of label propagation, on rows
    # short (registers), medium (shared-memory hash) and long (hub kernel)
    graphs = [graphgen.random_connected(500, 3000, seed=11, wmax=7),
              graphgen.planted(4, block_n=400, avg_deg=16, cross=6),
              graphgen.rhg(2, 1 << 14, 24.0),
              graphgen.rmat_kcore(2, scale=14, k=6),
              # rows of about 200-300 arcs on both sides of the warp kernel's
              # row limit, every label distinct in the first half-sweep
              graphgen.random_gnp(700, 0.36, seed=12, wmax=50),
              # many rows of 1-3 arcs packed into one batch
              graphgen.random_connected(5000, 1500, seed=13, wmax=4),
              # weights near 2^30: a label's total in a row passes 2^31
              graphgen.random_gnp(300, 0.1, seed=14, wmax=1 << 30)]
    # a star with a 3000-arc hub plus a ring, weights 1..9
    rng = np.random.default_rng(5)
    hub_u = np.zeros(3000, dtype=np.int64)
    hub_v = np.arange(1, 3001)
    ring_u = np.arange(1, 3001)
    ring_v = np.roll(ring_u, 1)
    u = np.concatenate([hub_u, ring_u])
    v = np.concatenate([hub_v, ring_v])
    graphs.append(graphgen.from_edges(3001, u, v, rng.integers(1, 10, size=len(u))))
    # a pure star: one row holds half of all arcs
    graphs.append(graphgen.from_edges(2001, np.zeros(2000, dtype=np.int64), np.arange(1, 2001),
                                      rng.integers(1, 10, size=2000)))
    for k, g in enumerate(graphs):
        with mc.Graph(*g) as G:
            lab = G.label_prop(iters, seed=77 + k)
        assert (lab == oracle.label_prop(*g, iters, 77 + k)).all(), k


@pytest.mark.parametrize("seed", range(4))
def test_lp_bound_planted(mc, seed):
    # the LP bound keeps lambda exact and finds the planted cut
    g = graphgen.planted(seed)
    ref, _, _ = oracle.noi(*g)
    with mc.Graph(*g) as G:
        res = G.min_cut(mc.options(bound=mc.MC_BOUND_LP))
    check_cut(mc, g, res, ref)
    assert res.stats["bound_initial"] >= ref


def test_lp_bound_lambda_unchanged(mc):
    for g in (graphgen.rhg(3, 1 << 16, 32.0), graphgen.rmat_kcore(3, scale=16),
              graphgen.random_connected(4000, 30000, seed=3, wmax=20)):
        ref, _, _ = oracle.noi(*g)
        with mc.Graph(*g) as G:
            res = G.min_cut(mc.options(bound=mc.MC_BOUND_LP, lp_iters=3))
        check_cut(mc, g, res, ref)


def test_injected_allocation_failures(mc):
    # host-side fault injection: every device allocation of graph creation,
    # solve and batch in turn fails; each call reports MC_ENOMEM, leaves
    # nothing behind, and the next call works
    g = graphgen.random_connected(300, 900, seed=5, wmax=5)
    ref = oracle.stoer_wagner(*g)[0]
    b = graphgen.batch(3, G=16)
    bref = [oracle.noi(*graphgen.batch_graph(b, k))[0] for k in range(16)]
    failures = 0
    try:
        for k in range(64):
            mc.test_fail_alloc_after(k)
            try:
                with mc.Graph(*g) as G:
                    res = G.min_cut(mc.options(bound=1))
                    assert res.lam == ref
                lam = mc.batch_min_cut(*b)[0]
                assert list(lam) == bref
            except mc.MinCutError as e:
                assert e.code == mc.MC_ENOMEM
                failures += 1
            mc.test_fail_alloc_after(-1)
            with mc.Graph(*g) as G:
                assert G.min_cut().lam == ref
    finally:
        mc.test_fail_alloc_after(-1)
    assert failures > 10
