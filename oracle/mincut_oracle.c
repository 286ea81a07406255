/*
 * mincut_oracle.c -- plain, slow, obviously-correct CPU oracle for the exact
 * global minimum cut of an undirected graph with non-negative integer weights.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  The product path (the CUDA
 * library) shares no code, header, table or helper with this file.
 *
 * Everything is single-threaded, int64 throughout, and written as the paper
 * (Henzinger, Noe, Schulz, "Shared-memory Exact Minimum Cuts") states it:
 *
 *   orc_cut_weight     Sec. 2.1 definition of the capacity c(A) of a cut.
 *   orc_degrees        Sec. 2.1 weighted degree; trivial cut / delta bound.
 *   orc_brute_force    Sec. 2.1 definition of lambda(G): minimum over all
 *                      proper non-empty A, enumerated in Gray-code order.
 *   orc_stoer_wagner   Stoer-Wagner maximum-adjacency phases (Sec. 2.2,
 *                      related work); an independent exact algorithm.
 *   orc_noi            Sequential NOI: repeat CAPFOREST (Appendix Alg. 3)
 *                      with the priority queue capped at lambda-hat
 *                      (Sec. 3.1.2, Lemma 1) and contract (Sec. 2.1), keeping
 *                      the side as in Sec. 3.3.
 *   orc_capforest_round  one capped CAPFOREST scan (Appendix Alg. 3) and the
 *                      unions it marks: one round of orc_noi on its own.
 *   orc_matula         Matula's (2+eps)-approximation: the same loop marking
 *                      at (1/2 - eps) times the minimum degree each round
 *                      (Sec. 2.2, Sec. 3.1.1).
 *   orc_contract       Sec. 2.1 edge contraction G/(u,v) applied to every
 *                      block of a vertex labelling at once.
 *   orc_label_prop     label propagation as used by VieCut (Sec. 2.3); the
 *                      paper gives no rule, the reading used is stated below.
 *   orc_pr_tests       Padberg-Rinaldi local contraction tests (Sec. 2.2
 *                      related work, used by VieCut in Sec. 2.3); the paper
 *                      does not state them, the reading used is stated below.
 *
 * Conventions shared with every caller:
 *   input graphs are symmetric CSR (row_ptr[n+1], col[], w[] as int32);
 *   self-loops and zero weights are ignored, parallel arcs are summed;
 *   a side is a uint8 array with side[v] = 1 iff v is NOT on vertex 0's side.
 *
 * Pins (tests/test_oracle_*.py): closed forms (K_n, C_n, trees, planted
 * cliques, disconnected graphs), brute force vs Stoer-Wagner vs NOI on
 * thousands of random tiny graphs, capped vs uncapped NOI, contraction
 * preserving the weight of every cut that does not split a block; Matula's
 * guarantee lambda <= cut <= lambda / (1/2 - eps) against brute force, its
 * side re-weighed, and exactness wherever lambda = delta.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;
typedef uint64_t u64;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOPROGRESS (-3)

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea, Flood 2014; constants as published by Vigna).   */
/* Used only to pick start vertices and the label-propagation parity split. */
u64 orc_splitmix64(u64 x)
{
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* ------------------------------------------------------------------------ */
/* A canonical weighted graph: rows sorted by neighbour, no self-loops, no   */
/* zero weights, parallel arcs summed, int64 weights.                       */
typedef struct {
    int n;
    i64 arcs;
    i64 *rp;   /* n+1 */
    int *col;  /* arcs */
    i64 *w;    /* arcs */
} ograph;

static void og_free(ograph *g)
{
    free(g->rp); free(g->col); free(g->w);
    memset(g, 0, sizeof(*g));
}

typedef struct { int u, v; i64 w; } otriple;

static int cmp_triple(const void *a, const void *b)
{
    const otriple *x = (const otriple *)a, *y = (const otriple *)b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/* Build a canonical graph on n vertices from a list of arcs (both directions
 * present).  Sorting by (u, v) and summing runs is the plain definition of
 * merging parallel edges (Sec. 2.1, contraction). */
static int og_from_triples(int n, otriple *t, i64 cnt, ograph *out)
{
    i64 k, m = 0;
    out->n = n;
    out->rp = (i64 *)calloc((size_t)n + 1, sizeof(i64));
    if (!out->rp) return ORC_ENOMEM;
    if (cnt > 0) qsort(t, (size_t)cnt, sizeof(otriple), cmp_triple);
    for (k = 0; k < cnt; ++k) {
        if (m > 0 && t[m - 1].u == t[k].u && t[m - 1].v == t[k].v) {
            t[m - 1].w += t[k].w;
        } else {
            t[m++] = t[k];
        }
    }
    out->arcs = m;
    out->col = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    out->w = (i64 *)malloc(sizeof(i64) * (size_t)(m > 0 ? m : 1));
    if (!out->col || !out->w) { og_free(out); return ORC_ENOMEM; }
    for (k = 0; k < m; ++k) {
        out->rp[t[k].u + 1]++;
        out->col[k] = t[k].v;
        out->w[k] = t[k].w;
    }
    for (k = 0; k < n; ++k) out->rp[k + 1] += out->rp[k];
    return ORC_OK;
}

static int og_from_csr(int n, const int32_t *rp, const int32_t *col,
                       const int32_t *w, ograph *out)
{
    i64 a, cnt = 0, arcs = rp[n];
    int u, rc;
    otriple *t = (otriple *)malloc(sizeof(otriple) * (size_t)(arcs > 0 ? arcs : 1));
    if (!t) return ORC_ENOMEM;
    for (u = 0; u < n; ++u) {
        for (a = rp[u]; a < rp[u + 1]; ++a) {
            if (col[a] == u || w[a] <= 0) continue; /* self-loop / zero weight */
            t[cnt].u = u; t[cnt].v = col[a]; t[cnt].w = w[a];
            ++cnt;
        }
    }
    rc = og_from_triples(n, t, cnt, out);
    free(t);
    return rc;
}

static int check_csr(int n, const int32_t *rp, const int32_t *col)
{
    int u;
    i64 a;
    if (n < 1 || rp[0] != 0) return ORC_EINVAL;
    for (u = 0; u < n; ++u)
        if (rp[u + 1] < rp[u]) return ORC_EINVAL;
    for (a = 0; a < rp[n]; ++a)
        if (col[a] < 0 || col[a] >= n) return ORC_EINVAL;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: c(A) = sum of c(u,v) over edges with exactly one end in A.      */
/* Each undirected edge appears as two arcs, so the arc sum is halved.       */
i64 orc_cut_weight(int n, const int32_t *rp, const int32_t *col,
                   const int32_t *w, const uint8_t *side)
{
    i64 s = 0, a;
    int u;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    for (u = 0; u < n; ++u)
        for (a = rp[u]; a < rp[u + 1]; ++a)
            if (col[a] != u && w[a] > 0 && (side[u] != 0) != (side[col[a]] != 0))
                s += w[a];
    return s / 2;
}

/* Sec. 2.1: weighted degree = sum of incident edge weights (self-loops are   */
/* not edges of a cut and are skipped).                                       */
int orc_degrees(int n, const int32_t *rp, const int32_t *col,
                const int32_t *w, i64 *deg)
{
    int u;
    i64 a;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    for (u = 0; u < n; ++u) {
        deg[u] = 0;
        for (a = rp[u]; a < rp[u + 1]; ++a)
            if (col[a] != u && w[a] > 0) deg[u] += w[a];
    }
    return ORC_OK;
}

/* Put the side into the canonical polarity: vertex 0 on side 0. */
static void canon_side(int n, uint8_t *side)
{
    int v;
    if (side[0]) for (v = 0; v < n; ++v) side[v] = (uint8_t)!side[v];
}

/* ------------------------------------------------------------------------ */
/* Brute force over the definition of lambda(G), Sec. 2.1.                   */
/* Vertex n-1 stays on side 0; the other n-1 vertices run through all        */
/* 2^(n-1) - 1 non-empty subsets in Gray-code order, so each step flips one  */
/* vertex and the cut changes by that vertex's arcs only.                    */
i64 orc_brute_force(int n, const int32_t *rp, const int32_t *col,
                    const int32_t *w, uint8_t *side_out)
{
    ograph g;
    uint8_t *side;
    u64 k, total, best_mask = 0;
    i64 cur = 0, best = -1, a;
    int v;
    if (n < 2 || n > 26) return ORC_EINVAL;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    side = (uint8_t *)calloc((size_t)n, 1);
    total = (u64)1 << (n - 1);
    for (k = 1; k < total; ++k) {
        v = __builtin_ctzll(k); /* Gray code: bit v flips between k-1 and k */
        for (a = g.rp[v]; a < g.rp[v + 1]; ++a)
            cur += (side[g.col[a]] == side[v]) ? g.w[a] : -g.w[a];
        side[v] ^= 1;
        if (best < 0 || cur < best) { best = cur; best_mask = k ^ (k >> 1); }
    }
    if (side_out) {
        for (v = 0; v < n; ++v) side_out[v] = (uint8_t)((v < n - 1) && ((best_mask >> v) & 1));
        canon_side(n, side_out);
    }
    free(side);
    og_free(&g);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Addressable binary max-heap on (key, -index), 0-based: children of slot i */
/* are 2i+1 and 2i+2 (the paper's 2i, 2i+1 are 1-based, Sec. 3.1.3).          */
typedef struct {
    int size;
    int *heap; /* slot -> vertex */
    int *pos;  /* vertex -> slot or -1 */
    i64 *key;  /* vertex -> key */
} oheap;

static int oh_init(oheap *h, int n)
{
    int v;
    h->size = 0;
    h->heap = (int *)malloc(sizeof(int) * (size_t)n);
    h->pos = (int *)malloc(sizeof(int) * (size_t)n);
    h->key = (i64 *)malloc(sizeof(i64) * (size_t)n);
    if (!h->heap || !h->pos || !h->key) return ORC_ENOMEM;
    for (v = 0; v < n; ++v) h->pos[v] = -1;
    return ORC_OK;
}

static void oh_free(oheap *h)
{
    free(h->heap); free(h->pos); free(h->key);
}

/* a outranks b: larger key, ties to the smaller vertex index */
static int oh_above(const oheap *h, int a, int b)
{
    if (h->key[a] != h->key[b]) return h->key[a] > h->key[b];
    return a < b;
}

static void oh_swap(oheap *h, int i, int j)
{
    int t = h->heap[i];
    h->heap[i] = h->heap[j];
    h->heap[j] = t;
    h->pos[h->heap[i]] = i;
    h->pos[h->heap[j]] = j;
}

static void oh_up(oheap *h, int i)
{
    while (i > 0) {
        int p = (i - 1) / 2;
        if (!oh_above(h, h->heap[i], h->heap[p])) break;
        oh_swap(h, i, p);
        i = p;
    }
}

static void oh_down(oheap *h, int i)
{
    for (;;) {
        int l = 2 * i + 1, r = l + 1, b = i;
        if (l < h->size && oh_above(h, h->heap[l], h->heap[b])) b = l;
        if (r < h->size && oh_above(h, h->heap[r], h->heap[b])) b = r;
        if (b == i) break;
        oh_swap(h, i, b);
        i = b;
    }
}

/* insert v with key k, or raise its key to k if k is larger */
static void oh_raise(oheap *h, int v, i64 k)
{
    if (h->pos[v] < 0) {
        h->key[v] = k;
        h->heap[h->size] = v;
        h->pos[v] = h->size++;
        oh_up(h, h->pos[v]);
    } else if (k > h->key[v]) {
        h->key[v] = k;
        oh_up(h, h->pos[v]);
    }
}

static int oh_pop(oheap *h)
{
    int v = h->heap[0];
    h->pos[v] = -1;
    if (--h->size > 0) {
        h->heap[0] = h->heap[h->size];
        h->pos[h->heap[0]] = 0;
        oh_down(h, 0);
    }
    return v;
}

/* ------------------------------------------------------------------------ */
/* Union-find with path halving (plain, sequential).                          */
static int uf_find(int *p, int x)
{
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/* link the larger root below the smaller one */
static int uf_union(int *p, int a, int b)
{
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return 0;
    if (a < b) p[b] = a; else p[a] = b;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Stoer-Wagner: n-1 maximum-adjacency phases on the current super-vertices   */
/* (union-find roots).  In each phase the last vertex t added has key         */
/* w(t, V \ t), the "cut of the phase"; the best such cut is the minimum cut; */
/* then t is merged into the second-to-last vertex s.                          */
i64 orc_stoer_wagner(int n, const int32_t *rp, const int32_t *col,
                     const int32_t *w, uint8_t *side_out)
{
    ograph g;
    oheap h;
    int *par = NULL, *next = NULL, *tail = NULL, *inA = NULL, *best_set = NULL;
    int v, phase, roots, best_root_count = 0;
    i64 best = -1;
    if (n < 2) return ORC_EINVAL;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    if (oh_init(&h, n) != ORC_OK) return ORC_ENOMEM;
    par = (int *)malloc(sizeof(int) * (size_t)n);
    next = (int *)malloc(sizeof(int) * (size_t)n);
    tail = (int *)malloc(sizeof(int) * (size_t)n);
    inA = (int *)malloc(sizeof(int) * (size_t)n);
    best_set = (int *)malloc(sizeof(int) * (size_t)n);
    for (v = 0; v < n; ++v) { par[v] = v; next[v] = -1; tail[v] = v; }
    roots = n;
    for (phase = 0; roots > 1; ++phase) {
        int s = -1, t = -1, x;
        i64 cut_of_phase = 0;
        for (v = 0; v < n; ++v) inA[v] = 0;
        for (v = 0; v < n; ++v)
            if (par[v] == v) oh_raise(&h, v, 0);
        while (h.size > 0) {
            int m;
            x = oh_pop(&h);
            inA[x] = 1;
            s = t; t = x;
            cut_of_phase = h.key[x];
            for (m = x; m >= 0; m = next[m]) {
                i64 a;
                for (a = g.rp[m]; a < g.rp[m + 1]; ++a) {
                    int y = uf_find(par, g.col[a]);
                    if (y == x || inA[y]) continue;
                    oh_raise(&h, y, (h.pos[y] < 0 ? 0 : h.key[y]) + g.w[a]);
                }
            }
        }
        if (best < 0 || cut_of_phase < best) {
            int m;
            best = cut_of_phase;
            best_root_count = 0;
            for (m = t; m >= 0; m = next[m]) best_set[best_root_count++] = m;
        }
        /* merge t into s: root stays the smaller index, member lists join */
        {
            int a = s < t ? s : t, b = s < t ? t : s;
            par[b] = a;
            next[tail[a]] = b;
            tail[a] = tail[b];
        }
        --roots;
    }
    if (side_out) {
        memset(side_out, 0, (size_t)n);
        for (v = 0; v < best_root_count; ++v) side_out[best_set[v]] = 1;
        canon_side(n, side_out);
    }
    oh_free(&h);
    free(par); free(next); free(tail); free(inA); free(best_set);
    og_free(&g);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Contraction of every block of a labelling at once (Sec. 2.1): block ids    */
/* lab[v] in [0, nc); arcs inside a block vanish, parallel arcs are summed.   */
static int og_contract(const ograph *g, const int *lab, int nc, ograph *out)
{
    i64 a, cnt = 0;
    int u, rc;
    otriple *t = (otriple *)malloc(sizeof(otriple) * (size_t)(g->arcs > 0 ? g->arcs : 1));
    if (!t) return ORC_ENOMEM;
    for (u = 0; u < g->n; ++u)
        for (a = g->rp[u]; a < g->rp[u + 1]; ++a) {
            int x = lab[u], y = lab[g->col[a]];
            if (x == y) continue;
            t[cnt].u = x; t[cnt].v = y; t[cnt].w = g->w[a];
            ++cnt;
        }
    rc = og_from_triples(nc, t, cnt, out);
    free(t);
    return rc;
}

/* Public form: contract an int32 CSR by labels; writes the canonical CSR of  */
/* the contracted graph (rows sorted, int64 weights).  out_rp has nc+1 slots, */
/* out_col/out_w have at least rp[n] slots.  Returns the arc count.           */
i64 orc_contract(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
                 const int32_t *lab, int nc, i64 *out_rp, int32_t *out_col,
                 i64 *out_w)
{
    ograph g, c;
    i64 a;
    int v, rc;
    if (check_csr(n, rp, col) != ORC_OK || nc < 1) return ORC_EINVAL;
    for (v = 0; v < n; ++v)
        if (lab[v] < 0 || lab[v] >= nc) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    rc = og_contract(&g, lab, nc, &c);
    og_free(&g);
    if (rc != ORC_OK) return rc;
    for (v = 0; v <= nc; ++v) out_rp[v] = c.rp[v];
    for (a = 0; a < c.arcs; ++a) { out_col[a] = c.col[a]; out_w[a] = c.w[a]; }
    a = c.arcs;
    og_free(&c);
    return a;
}

/* ------------------------------------------------------------------------ */
/* Sequential NOI with the lambda-hat-capped priority queue.                  */
/*                                                                            */
/* One round is CAPFOREST (Appendix Alg. 3) from a start vertex:              */
/*   pop x with the largest key;                                              */
/*   alpha += c(x) - 2 r(x); lambda-hat = min(lambda-hat, alpha) while the     */
/*     scanned set S is a proper subset (alpha = c(S));                        */
/*   for every arc (x, y, c) to an unscanned y:                                */
/*     if r(y) < lambda-hat <= r(y) + c, mark (x, y) for contraction;          */
/*     r(y) += c;  key(y) = r(y)  (uncapped)  or                               */
/*                 key(y) = max(key(y), min(r(y), lambda-hat))  (capped);      */
/*   mark x scanned.                                                           */
/* Keys are never lowered: Sec. 3.1.2 / Sec. 3.2 leave priorities that already */
/* reached lambda-hat alone, and Lemma 1's proof only ever lowers edge weights */
/* so that r stops at the cap.                                                 */
/* Then the marked edges are contracted (Sec. 2.1) and lambda-hat drops to the */
/* minimum weighted degree of the contracted graph if that is smaller          */
/* (Sec. 3.2, parallel graph contraction).  Each improvement of lambda-hat     */
/* records its side through the map original vertex -> current vertex         */
/* (Sec. 3.3).  Rounds repeat until one vertex is left or lambda-hat is 0.     */
/* A round that marks nothing must have lowered lambda-hat (Sec. 2.2: a full   */
/* CAPFOREST with lambda-hat <= delta marks an edge unless lambda-hat dropped  */
/* inside the round); otherwise the oracle reports ORC_ENOPROGRESS.            */
/*                                                                            */
/* With approx_milli = a in [1, 500] the same loop is Matula's                */
/* (2+eps)-approximation as Sec. 3.1.1 describes it: each round marks at the  */
/* threshold t = min(lambda-hat, ceil(a * delta / 1000)), (1/2 - eps) times   */
/* the current minimum degree, instead of at lambda-hat; lambda-hat keeps the */
/* best real cut (degrees, alpha values below t).  a = 0 is the exact loop.   */
static i64 noi_loop(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
                    int capped, int approx_milli, u64 seed, uint8_t *side_out, int32_t *rounds_out)
{
    ograph g;
    int *map = NULL, *lab = NULL, *par = NULL, *scanned = NULL, *order = NULL;
    i64 *r = NULL, *deg = NULL;
    uint8_t *best_side = NULL;
    i64 lam;
    int v, rounds = 0, rc = ORC_OK;
    if (n < 2) return ORC_EINVAL;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    map = (int *)malloc(sizeof(int) * (size_t)n);
    lab = (int *)malloc(sizeof(int) * (size_t)n);
    par = (int *)malloc(sizeof(int) * (size_t)n);
    scanned = (int *)malloc(sizeof(int) * (size_t)n);
    order = (int *)malloc(sizeof(int) * (size_t)n);
    r = (i64 *)malloc(sizeof(i64) * (size_t)n);
    deg = (i64 *)malloc(sizeof(i64) * (size_t)n);
    best_side = (uint8_t *)calloc((size_t)n, 1);
    if (!map || !lab || !par || !scanned || !order || !r || !deg || !best_side) {
        rc = ORC_ENOMEM;
        goto done;
    }
    for (v = 0; v < n; ++v) map[v] = v;

    /* lambda-hat starts at the trivial cut of a minimum-degree vertex (Sec. 2.1) */
    {
        i64 a;
        int arg = 0;
        for (v = 0; v < g.n; ++v) {
            deg[v] = 0;
            for (a = g.rp[v]; a < g.rp[v + 1]; ++a) deg[v] += g.w[a];
            if (deg[v] < deg[arg]) arg = v;
        }
        lam = deg[arg];
        for (v = 0; v < n; ++v) best_side[v] = (uint8_t)(v == arg);
    }

    while (g.n >= 2 && lam > 0) {
        oheap h;
        int nS = 0, start, x, nc;
        i64 alpha = 0, marked = 0, thr = lam, thr_at_start;
        if (approx_milli > 0) {
            i64 dmin = deg[0], t;
            for (v = 1; v < g.n; ++v)
                if (deg[v] < dmin) dmin = deg[v];
            t = dmin / 1000 * approx_milli + (dmin % 1000 * approx_milli + 999) / 1000;
            if (t < 1) t = 1;
            if (t < thr) thr = t;
        }
        thr_at_start = thr;
        if (oh_init(&h, g.n) != ORC_OK) { rc = ORC_ENOMEM; goto done; }
        for (v = 0; v < g.n; ++v) { par[v] = v; scanned[v] = 0; r[v] = 0; }
        start = (int)(orc_splitmix64(seed ^ (u64)rounds) % (u64)g.n);
        oh_raise(&h, start, 0);
        while (h.size > 0) {
            i64 a;
            x = oh_pop(&h);
            alpha += deg[x] - 2 * r[x];
            order[nS++] = x;
            if (nS < g.n && alpha < thr) {
                int k;
                lam = alpha;
                thr = alpha;
                for (v = 0; v < g.n; ++v) lab[v] = 0;
                for (k = 0; k < nS; ++k) lab[order[k]] = 1;
                for (v = 0; v < n; ++v) best_side[v] = (uint8_t)lab[map[v]];
            }
            for (a = g.rp[x]; a < g.rp[x + 1]; ++a) {
                int y = g.col[a];
                i64 c = g.w[a];
                if (scanned[y]) continue;
                if (r[y] < thr && thr <= r[y] + c) marked += uf_union(par, x, y);
                r[y] += c;
                if (capped) {
                    i64 k = r[y] < thr ? r[y] : thr;
                    oh_raise(&h, y, k);
                } else {
                    oh_raise(&h, y, r[y]);
                }
            }
            scanned[x] = 1;
        }
        oh_free(&h);
        ++rounds;
        if (lam == 0) break;
        if (marked == 0) {
            if (thr < thr_at_start) continue;
            rc = ORC_ENOPROGRESS;
            goto done;
        }
        /* block ids in order of the smallest member */
        nc = 0;
        for (v = 0; v < g.n; ++v) lab[v] = -1;
        for (v = 0; v < g.n; ++v) {
            int root = uf_find(par, v);
            if (lab[root] < 0) lab[root] = nc++;
            lab[v] = lab[root];
        }
        {
            ograph c;
            i64 a;
            int arg = 0;
            if (og_contract(&g, lab, nc, &c) != ORC_OK) { rc = ORC_ENOMEM; goto done; }
            og_free(&g);
            g = c;
            for (v = 0; v < n; ++v) map[v] = lab[map[v]];
            for (v = 0; v < g.n; ++v) {
                deg[v] = 0;
                for (a = g.rp[v]; a < g.rp[v + 1]; ++a) deg[v] += g.w[a];
                if (deg[v] < deg[arg]) arg = v;
            }
            if (g.n >= 2 && deg[arg] < lam) {
                lam = deg[arg];
                for (v = 0; v < n; ++v) best_side[v] = (uint8_t)(map[v] == arg);
            }
        }
    }
    if (side_out) {
        memcpy(side_out, best_side, (size_t)n);
        canon_side(n, side_out);
    }
done:
    if (rounds_out) *rounds_out = rounds;
    free(map); free(lab); free(par); free(scanned); free(order);
    free(r); free(deg); free(best_side);
    og_free(&g);
    return rc == ORC_OK ? lam : rc;
}

i64 orc_noi(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
            int capped, u64 seed, uint8_t *side_out, int32_t *rounds_out)
{
    return noi_loop(n, rp, col, w, capped, 0, seed, side_out, rounds_out);
}

/* Matula's (2+eps)-approximation (Sec. 2.2, Sec. 3.1.1): a real cut of      */
/* weight at most 1000 / approx_milli times lambda; approx_milli in [1, 500]. */
i64 orc_matula(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
               int approx_milli, u64 seed, uint8_t *side_out, int32_t *rounds_out)
{
    if (approx_milli < 1 || approx_milli > 500) return ORC_EINVAL;
    return noi_loop(n, rp, col, w, 1, approx_milli, seed, side_out, rounds_out);
}

/* One capped CAPFOREST scan (Appendix Alg. 3) from `start` against the      */
/* bound lam: the steps of one orc_noi round, on its own.  lab_out[v] = the   */
/* smallest vertex of v's block of marked edges; returns lambda-hat after the */
/* scan (lowered by alpha while the scanned set is a proper subset).          */
i64 orc_capforest_round(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
                        i64 lam, int start, int32_t *lab_out)
{
    ograph g;
    oheap h;
    int *par = NULL, *scanned = NULL;
    i64 *r = NULL, *deg = NULL, alpha = 0;
    int v, nS = 0, rc = ORC_OK;
    if (n < 1 || start < 0 || start >= n || lam < 0) return ORC_EINVAL;
    if (check_csr(n, rp, col) != ORC_OK) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    par = (int *)malloc(sizeof(int) * (size_t)n);
    scanned = (int *)calloc((size_t)n, sizeof(int));
    r = (i64 *)calloc((size_t)n, sizeof(i64));
    deg = (i64 *)calloc((size_t)n, sizeof(i64));
    if (!par || !scanned || !r || !deg || oh_init(&h, n) != ORC_OK) {
        free(par); free(scanned); free(r); free(deg);
        og_free(&g);
        return ORC_ENOMEM;
    }
    for (v = 0; v < n; ++v) {
        i64 a;
        par[v] = v;
        for (a = g.rp[v]; a < g.rp[v + 1]; ++a) deg[v] += g.w[a];
    }
    oh_raise(&h, start, 0);
    while (h.size > 0) {
        i64 a;
        const int x = oh_pop(&h);
        alpha += deg[x] - 2 * r[x];
        ++nS;
        if (nS < n && alpha < lam) lam = alpha;
        for (a = g.rp[x]; a < g.rp[x + 1]; ++a) {
            const int y = g.col[a];
            const i64 c = g.w[a];
            if (scanned[y]) continue;
            if (r[y] < lam && lam <= r[y] + c) uf_union(par, x, y);
            r[y] += c;
            oh_raise(&h, y, r[y] < lam ? r[y] : lam);
        }
        scanned[x] = 1;
    }
    for (v = 0; v < n; ++v) lab_out[v] = uf_find(par, v);
    oh_free(&h);
    free(par); free(scanned); free(r); free(deg);
    og_free(&g);
    return rc == ORC_OK ? lam : rc;
}

/* ------------------------------------------------------------------------ */
/* Label propagation (VieCut, Sec. 2.3; rule of Raghavan et al.).  The paper  */
/* gives no details; the reading used throughout this project is:             */
/*   labels start as the vertex ids;                                          */
/*   each of `iters` sweeps has two half-sweeps p = 0, 1; in half-sweep p the  */
/*   vertices with parity(seed, sweep, v) == p take, all at once from the      */
/*   labels as they stand, the label l maximising the total weight of arcs     */
/*   to neighbours labelled l (ties to the smallest l; no neighbours: keep);   */
/*   parity(seed, s, v) = splitmix64(seed ^ splitmix64(((u64)s << 32) | v)) & 1 */
int orc_label_prop(int n, const int32_t *rp, const int32_t *col,
                   const int32_t *w, int iters, u64 seed, int32_t *labels)
{
    ograph g;
    int32_t *cur, *nxt;
    i64 *acc;
    int *touched;
    int it, p, v;
    if (check_csr(n, rp, col) != ORC_OK || iters < 0) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    acc = (i64 *)calloc((size_t)n, sizeof(i64));
    touched = (int *)malloc(sizeof(int) * (size_t)n);
    for (v = 0; v < n; ++v) cur[v] = v;
    for (it = 0; it < iters; ++it) {
        for (p = 0; p < 2; ++p) {
            for (v = 0; v < n; ++v) {
                u64 h = orc_splitmix64(seed ^ orc_splitmix64(((u64)(uint32_t)it << 32) | (u64)(uint32_t)v));
                i64 a, bw = -1;
                int nt = 0, k, bl = cur[v];
                nxt[v] = cur[v];
                if ((int)(h & 1) != p) continue;
                if (g.rp[v] == g.rp[v + 1]) continue;
                for (a = g.rp[v]; a < g.rp[v + 1]; ++a) {
                    int l = cur[g.col[a]];
                    if (acc[l] == 0) touched[nt++] = l;
                    acc[l] += g.w[a];
                }
                for (k = 0; k < nt; ++k) {
                    int l = touched[k];
                    if (acc[l] > bw || (acc[l] == bw && l < bl)) { bw = acc[l]; bl = l; }
                }
                for (k = 0; k < nt; ++k) acc[touched[k]] = 0;
                nxt[v] = bl;
            }
            memcpy(cur, nxt, sizeof(int32_t) * (size_t)n);
        }
    }
    memcpy(labels, cur, sizeof(int32_t) * (size_t)n);
    free(cur); free(nxt); free(acc); free(touched);
    og_free(&g);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Padberg-Rinaldi tests.  The paper cites them (Sec. 2.2 related work,       */
/* Sec. 2.3) without stating them; the reading used, with d() the weighted    */
/* degree and lam the current bound, is that edge {u, v} may be contracted    */
/* when                                                                       */
/*   PR1: c(u,v) >= lam                                                        */
/*   PR2: 2 c(u,v) > min(d(u), d(v))                                           */
/*   PR3: some common neighbour w has 2(c(u,v) + c(u,w)) > d(u) and           */
/*        2(c(u,v) + c(v,w)) > d(v)                                            */
/*   PR4: c(u,v) + sum over common neighbours w of min(c(u,w), c(v,w)) >= lam   */
/* PR2 and PR3 are strict because every edge that passes is contracted at      */
/* once: with ">=" a path of weight-w edges through degree-2w vertices would   */
/* be contracted whole and its cut of weight w lost.  With level >= 2 one more */
/* rule covers the tie PR2 leaves out: a vertex u with exactly two neighbours  */
/* joined by equal weights c is united with the smaller of the two.  Any cut   */
/* below delta = min degree <= 2c crosses a maximal path of such vertices at   */
/* most once, can be slid along it without changing its weight, and the path's */
/* k inner vertices unite at most k of its k+1 edges, so one stays open;      */
/* a graph that is one such cycle has lambda = delta.  `level` selects the     */
/* tests 1..level.  labels[v] receives the smallest vertex of v's block in the  */
/* graph of all passing edges.                                                 */
int orc_pr_tests(int n, const int32_t *rp, const int32_t *col, const int32_t *w,
                 i64 lam, int level, int32_t *labels)
{
    ograph g;
    i64 *deg, *cw;
    int *par;
    int u, v;
    i64 a, b;
    if (check_csr(n, rp, col) != ORC_OK || level < 0 || level > 4) return ORC_EINVAL;
    if (og_from_csr(n, rp, col, w, &g) != ORC_OK) return ORC_ENOMEM;
    deg = (i64 *)calloc((size_t)n, sizeof(i64));
    cw = (i64 *)calloc((size_t)n, sizeof(i64)); /* c(u, .) scattered for lookups */
    par = (int *)malloc(sizeof(int) * (size_t)n);
    for (u = 0; u < n; ++u) {
        par[u] = u;
        for (a = g.rp[u]; a < g.rp[u + 1]; ++a) deg[u] += g.w[a];
    }
    for (u = 0; u < n; ++u) {
        for (a = g.rp[u]; a < g.rp[u + 1]; ++a) cw[g.col[a]] = g.w[a];
        for (a = g.rp[u]; a < g.rp[u + 1]; ++a) {
            i64 c = g.w[a], md, pr4 = c;
            int ok = 0;
            v = g.col[a];
            md = deg[u] < deg[v] ? deg[u] : deg[v];
            if (level >= 1 && c >= lam) ok = 1;
            if (level >= 2 && 2 * c > md) ok = 1;
            if (level >= 3) {
                for (b = g.rp[v]; b < g.rp[v + 1]; ++b) {
                    int x = g.col[b];
                    i64 cux = cw[x], cvx = g.w[b];
                    if (x == u || cux == 0) continue;
                    if (2 * (c + cux) > deg[u] && 2 * (c + cvx) > deg[v]) ok = 1;
                    pr4 += cux < cvx ? cux : cvx;
                }
                if (level >= 4 && pr4 >= lam) ok = 1;
            }
            if (ok) uf_union(par, u, v);
        }
        for (a = g.rp[u]; a < g.rp[u + 1]; ++a) cw[g.col[a]] = 0;
    }
    if (level >= 2) {
        for (u = 0; u < n; ++u) {
            a = g.rp[u];
            if (g.rp[u + 1] - a == 2 && g.w[a] == g.w[a + 1])
                uf_union(par, u, g.col[a] < g.col[a + 1] ? g.col[a] : g.col[a + 1]);
        }
    }
    for (v = 0; v < n; ++v) labels[v] = uf_find(par, v);
    free(deg); free(cw); free(par);
    og_free(&g);
    return ORC_OK;
}
