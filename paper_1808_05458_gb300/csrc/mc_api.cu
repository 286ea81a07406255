// mc_api.cu -- the C ABI (include/mc.h) and the host driver of Alg. 2.
//
// Driver per round on the current graph G_C (Alg. 2, Sec. 3.3):
//   union-find reset -> Padberg-Rinaldi tests -> concurrent capped CAPFOREST
//   (Alg. 1) -> if nothing was united: one full CAPFOREST scan (Alg. 3) ->
//   contraction (Sec. 3.2) -> lambda-hat = min(lambda-hat, delta(G_C)).
// Every improvement of lambda-hat snapshots its side as a bitmap over the
// original vertices (Sec. 3.3): a scan's prefix for an alpha cut, the
// preimage of a contracted vertex for a degree cut.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "mc_internal.cuh"

using namespace mc;

struct mc_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    int n0 = 0;
    i64 arcs0 = 0;
    DevGraph G0, Ga, Gb;
    Work w;
    i64 delta0 = 0;
    int argmin0 = 0;
    i64 wmax0 = 0;          // largest arc weight of G0
    i64 two_arc_rows0 = 0;  // rows of G0 with exactly two arcs
    bool device_ptrs = false;
    bool complete = false;  // every buffer allocated and the input built
    std::vector<cudaEvent_t> events;  // phase-clock events, reused across calls
    // host input staging: a copy stream and one event per chunk, made on
    // first use and kept with the graph
    cudaStream_t copy = nullptr;
    cudaEvent_t ready[4] = {};
};

namespace {

struct Timer {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t s;
    explicit Timer(cudaStream_t s_) : s(s_) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    double ms() {
        float t = 0;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&t, a, b);
        cudaEventRecord(a, s);
        return t;
    }
};

// Phase times from events recorded at phase boundaries and read only once the
// call has synchronised at its end, so the timing adds no waits: each mark
// closes the interval since the previous mark and adds it to an accumulator
// (or drops it); spans add the time between two marks of their own.
struct PhaseClock {
    std::vector<cudaEvent_t> &pool;
    cudaStream_t s;
    std::vector<double *> dst;                       // accumulator per interval
    std::vector<std::pair<size_t, size_t>> span_ev;  // (begin, end) event indices
    std::vector<double *> span_dst;
    size_t used = 0;
    PhaseClock(std::vector<cudaEvent_t> &p, cudaStream_t s_) : pool(p), s(s_) { mark(nullptr); }
    size_t record() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        cudaEventRecord(pool[used], s);
        return used++;
    }
    void mark(double *acc) {
        record();
        dst.push_back(acc);
    }
    size_t span_begin() {
        const size_t i = record();
        dst.push_back(nullptr);
        return i;
    }
    void span_end(size_t b, double *acc) {
        const size_t e = record();
        dst.push_back(nullptr);
        span_ev.emplace_back(b, e);
        span_dst.push_back(acc);
    }
    // the last interval now (synchronises; for verbose output only)
    double last_ms() {
        float t = 0;
        cudaEventSynchronize(pool[used - 1]);
        cudaEventElapsedTime(&t, pool[used - 2], pool[used - 1]);
        return t;
    }
    void finish() {
        if (used) cudaEventSynchronize(pool[used - 1]);
        for (size_t i = 1; i < used; ++i)
            if (dst[i]) {
                float t = 0;
                cudaEventElapsedTime(&t, pool[i - 1], pool[i]);
                *dst[i] += t;
            }
        for (size_t k = 0; k < span_ev.size(); ++k) {
            float t = 0;
            cudaEventElapsedTime(&t, pool[span_ev[k].first], pool[span_ev[k].second]);
            *span_dst[k] += t;
        }
    }
};

void destroy_all(mc_graph *g) {
    if (!g) return;
    cudaStream_t s = g->stream;
    if (s) cudaStreamSynchronize(s);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    if (g->copy) {
        cudaStreamSynchronize(g->copy);
        cudaStreamDestroy(g->copy);
    }
    for (cudaEvent_t e : g->ready)
        if (e) cudaEventDestroy(e);
    graph_free(g->G0, s);
    graph_free(g->Ga, s);
    graph_free(g->Gb, s);
    work_free(g->w, s);
    if (s) cudaStreamDestroy(s);
    delete g;
}

// One destroyed graph per device is kept -- its stream, events and device
// buffers -- for the next graph created on that device with at most its
// vertex and arc counts (every buffer is sized by those two); a larger graph
// replaces it.  Not while the allocation fault-injection hook is armed.
struct ShellCache {
    std::mutex m;
    mc_graph *g[64] = {};
};
ShellCache g_shells;

mc_graph *take_shell(int dev, int n, i64 arcs) {
    if (dev < 0 || dev >= 64 || test_alloc_hook_armed()) return nullptr;
    std::lock_guard<std::mutex> lock(g_shells.m);
    mc_graph *c = g_shells.g[dev];
    if (!c || c->w.cap_n < n || c->w.cap_arcs < arcs) return nullptr;
    g_shells.g[dev] = nullptr;
    return c;
}

// true if g was kept (its work on the stream finished first)
bool park_shell(mc_graph *g) {
    if (!g->complete || g->device < 0 || g->device >= 64 || test_alloc_hook_armed()) return false;
    if (g->stream) cudaStreamSynchronize(g->stream);
    if (cudaGetLastError() != cudaSuccess) return false;
    mc_graph *old = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_shells.m);
        mc_graph *&slot = g_shells.g[g->device];
        if (slot && slot->w.cap_n >= g->w.cap_n && slot->w.cap_arcs >= g->w.cap_arcs) return false;
        old = slot;
        slot = g;
    }
    if (old) destroy_all(old);
    return true;
}

cudaStream_t pick_stream(mc_graph *g, const mc_options *o) {
    return (o && o->cuda_stream) ? static_cast<cudaStream_t>(o->cuda_stream) : g->stream;
}

int create_impl(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                int32_t flags, mc_graph **out) {
    if (!out || !row_ptr || n < 2) return MC_EINVAL;
    *out = nullptr;
    const bool dev = (flags & MC_DEVICE_PTRS) != 0;
    int device = 0;
    MC_CUDA(cudaGetDevice(&device));
    int arcs_raw = 0;
    if (dev) MC_CUDA(cudaMemcpy(&arcs_raw, row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost));
    else arcs_raw = row_ptr[n];
    if (arcs_raw < 0 || (arcs_raw > 0 && !col)) return MC_EINVAL;
    const i64 A = arcs_raw > 0 ? arcs_raw : 1;
    int rc = MC_OK;
    mc_graph *g = take_shell(device, n, A);
    if (g) {
        // a kept graph: its buffers are large enough; the input is built
        // into them below
        g->complete = false;
    } else {
        g = new mc_graph();
        g->device = device;
        cudaError_t e = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaStreamCreate");
            delete g;
            return MC_ECUDA;
        }
        if ((rc = work_alloc(g->w, n, A, g->stream)) != MC_OK || (rc = graph_alloc(g->G0, n, A, g->stream)) != MC_OK ||
            (rc = graph_alloc(g->Ga, n, A, g->stream)) != MC_OK || (rc = graph_alloc(g->Gb, n, A, g->stream)) != MC_OK) {
            destroy_all(g);
            return rc;
        }
    }
    g->device_ptrs = dev;
    g->n0 = n;
    cudaStream_t s = g->stream;
    const int *drp = row_ptr, *dcol = col, *dw = w;
    // host input: the raw arrays are staged in Ga (rp, src) and Gb (src);
    // the arcs go in kStageChunks chunks of whole rows on a copy stream, so
    // that each chunk is canonicalised while the next one is on the way (two
    // copy streams taking turns measured slower: creation 1.08 -> 1.15 ms)
    constexpr int kStageChunks = 4;
    StagedInput staged;
    int row_split[kStageChunks + 1];
    if (!dev) {
        cudaError_t e = cudaMemcpyAsync(g->Ga.rp, row_ptr, sizeof(int) * ((size_t)n + 1),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && arcs_raw > 0 && !g->copy)
            e = cudaStreamCreateWithFlags(&g->copy, cudaStreamNonBlocking);
        for (int k = 0; k < kStageChunks && e == cudaSuccess && arcs_raw > 0; ++k)
            if (!g->ready[k]) e = cudaEventCreateWithFlags(&g->ready[k], cudaEventDisableTiming);
        if (e == cudaSuccess && arcs_raw > 0) {
            // row splits at about equal arc counts (a search over the host
            // offsets; they are validated on the device before any chunk is
            // read)
            row_split[0] = 0;
            for (int k = 1; k < kStageChunks; ++k) {
                const i64 target = (i64)arcs_raw * k / kStageChunks;
                int lo = row_split[k - 1], hi = n;
                while (lo < hi) {
                    const int mid = lo + (hi - lo + 1) / 2;
                    if ((i64)row_ptr[mid] <= target) lo = mid; else hi = mid - 1;
                }
                row_split[k] = lo;
            }
            row_split[kStageChunks] = n;
            for (int k = 0; k < kStageChunks && e == cudaSuccess; ++k) {
                // clamped: offsets that fail the device check never reach a
                // build, but their copies must stay inside both buffers
                i64 a0 = k == 0 ? 0 : row_ptr[row_split[k]];
                i64 a1 = k == kStageChunks - 1 ? arcs_raw : row_ptr[row_split[k + 1]];
                a0 = a0 < 0 ? 0 : (a0 > arcs_raw ? arcs_raw : a0);
                a1 = a1 < a0 ? a0 : (a1 > arcs_raw ? arcs_raw : a1);
                cudaStream_t cs = g->copy;
                if (a1 > a0)
                    e = cudaMemcpyAsync(g->Ga.src + a0, col + a0, sizeof(int) * (size_t)(a1 - a0),
                                        cudaMemcpyHostToDevice, cs);
                if (e == cudaSuccess && a1 > a0 && w)
                    e = cudaMemcpyAsync(g->Gb.src + a0, w + a0, sizeof(int) * (size_t)(a1 - a0),
                                        cudaMemcpyHostToDevice, cs);
                if (e == cudaSuccess) e = cudaEventRecord(g->ready[k], cs);
            }
            staged.chunks = kStageChunks;
            staged.row_split = row_split;
            staged.ready = g->ready;
        }
        staged.arcs = arcs_raw;
        if (e != cudaSuccess) {
            set_cuda_error(e, "cudaMemcpyAsync(input)");
            destroy_all(g);  // waits for the copy stream
            return MC_ECUDA;
        }
        drp = g->Ga.rp;
        dcol = g->Ga.src;
        dw = w ? g->Gb.src : nullptr;
    }
    rc = canonicalize(n, drp, dcol, dw, (flags & MC_TRUST_INPUT) == 0, g->G0, g->w, s, dev ? nullptr : &staged);
    // on an early return canonicalize did not wait for every chunk
    if (rc != MC_OK && g->copy) cudaStreamSynchronize(g->copy);
    if (rc == MC_OK) rc = min_degree(g->G0, g->w, s);
    if (rc == MC_OK) rc = graph_stats(g->G0, g->w, s);
    if (rc == MC_OK) rc = status_read(g->w, s);
    if (rc == MC_OK) {
        g->delta0 = g->w.h_st->mindeg;
        g->argmin0 = g->w.h_st->argmin;
        g->wmax0 = g->w.h_st->count;
        g->two_arc_rows0 = g->w.h_st->count2;
        if (g->delta0 >= (1LL << 62)) rc = MC_EOVERFLOW;
    }
    if (rc != MC_OK) {
        destroy_all(g);
        return rc;
    }
    g->arcs0 = g->G0.arcs;
    g->complete = true;
    *out = g;
    return MC_OK;
}

// The bound phase: up to 8 levels of { LP sweeps -> contract the clusters ->
// lambda-hat = min(., delta) -> PR tests -> contract }, then the exact loop on
// what is left (at most kLpSmall vertices or no further clustering).  Runs on
// Ga / Gb, leaves G0 untouched.
// level 0 of the bound phase: `iters` label-propagation sweeps on G0, dense
// cluster ids in w.lab, the cluster graph in Ga (merged weights clamped to
// `clamp`), w.orig = each original vertex's cluster, the cluster graph's
// minimum degree in w.h_st; *nc = clusters (the graph is left alone when
// there are fewer than two)
int cluster_level0(mc_graph *g, int iters, u64 seed, i64 clamp, int *nc, cudaStream_t s) {
    Work &w = g->w;
    MC_TRY(label_prop(g->G0, w, iters, seed, w.lab, s));
    MC_TRY(compact_labels(w, g->n0, nc, s));
    if (*nc < 2) return MC_OK;
    MC_TRY(iota_i32(w.orig, g->n0, s));
    MC_TRY(round_reset(w, clamp, s));
    return contract_graph(g->G0, g->Ga, w, clamp, false, *nc, s, [&]() -> int {
        MC_TRY(orig_update(w, g->n0, s));
        return min_degree(g->Ga, w, s);
    });
}

// the learned proposer's sweep cut over the clusters of `cl` (a cluster graph
// whose vertices w.orig maps the original ones to): lowers lam, with its
// side, when the cut is below it.  A sweep cut below the contraction's clamp
// holds no clamped edge, so its weight is that of a real cut of G.
int proposer_on_clusters(mc_graph *g, Proposer &pp, const DevGraph &cl, i64 delta_cl, i64 &lam, bool verbose,
                         cudaStream_t s) {
    long long cut = 0;
    int k = 0;
    MC_TRY(proposer_forward(pp, cl, delta_cl, s));
    MC_TRY(proposer_sweep(pp, cl, g->w, &cut, &k, s));
    if (verbose)
        fprintf(stderr, "[mc] proposer on %d clusters: sweep cut %lld (k=%d), bound %lld\n", cl.n, cut, k,
                (long long)lam);
    if (cut < lam) {
        lam = cut;
        MC_TRY(side_from_rank(g->w, g->n0, k, true, s));
    }
    return MC_OK;
}

template <class Exact>
int lp_bound(mc_graph *g, const mc_options &o, i64 &lam, cudaStream_t s, bool verbose, i64 &bytes,
             Exact exact, Proposer *pp = nullptr) {
    Work &w = g->w;
    const int n0 = g->n0;
    constexpr int kLpSmall = 2048;
    const int iters = o.lp_iters > 0 ? o.lp_iters : 2;
    DevGraph cur = g->G0;
    DevGraph *nxt = &g->Ga;
    for (int level = 0; level < 8 && cur.n > kLpSmall && lam > 0; ++level) {
        MC_TRY(label_prop(cur, w, iters, o.seed ^ (0x9E37ULL * (u64)(level + 1)), w.lab, s));
        bytes += (cur.arcs * 12 + (i64)cur.n * 12) * 2 * iters;
        int nc = 0;
        MC_TRY(compact_labels(w, cur.n, &nc, s));
        if (verbose)
            fprintf(stderr, "[mc] bound level %d: n=%d arcs=%lld -> %d clusters\n", level, cur.n,
                    (long long)cur.arcs, nc);
        if (nc < 2 || (long long)nc * 10 > (long long)cur.n * 9) break;
        MC_TRY(round_reset(w, lam, s));
        MC_TRY(contract_graph(cur, *nxt, w, lam, false, nc, s, [&]() -> int {
            MC_TRY(orig_update(w, n0, s));
            return min_degree(*nxt, w, s);
        }));
        bytes += cur.arcs * 20;
        const i64 delta_cl = w.h_st->mindeg;
        if (delta_cl < lam) {
            lam = delta_cl;
            MC_TRY(side_from_vertex(w, n0, w.h_st->argmin, s));
        }
        cur = *nxt;
        nxt = (nxt == &g->Ga) ? &g->Gb : &g->Ga;
        // the learned proposer votes on the first level's clusters
        if (pp && level == 0) MC_TRY(proposer_on_clusters(g, *pp, cur, delta_cl, lam, verbose, s));
        // Padberg-Rinaldi on the cluster graph
        MC_TRY(round_start(w, cur.n, lam, s));
        MC_TRY(pr_tests_budget(cur, w, lam, 1, 4, 64, s));
        MC_TRY(status_read(w, s));
        if (w.h_st->unions > 0 && cur.n >= 2) {
            MC_TRY(contract_graph(cur, *nxt, w, lam, true, 0, s, [&]() -> int {
                MC_TRY(orig_update(w, n0, s));
                return min_degree(*nxt, w, s);
            }));
            if (nxt->n >= 2 && w.h_st->mindeg < lam) {
                lam = w.h_st->mindeg;
                MC_TRY(side_from_vertex(w, n0, w.h_st->argmin, s));
            }
            cur = *nxt;
            nxt = (nxt == &g->Ga) ? &g->Gb : &g->Ga;
        }
        if (verbose)
            fprintf(stderr, "[mc] bound level %d: after PR n=%d lam=%lld\n", level, cur.n, (long long)lam);
    }
    // the exact minimum cut of what is left is a cut of G as well
    if (cur.n >= 2 && cur.rp != g->G0.rp) MC_TRY(exact(cur, nxt));
    return MC_OK;
}

struct SolveOut {
    i64 lam = 0;
    mc_stats st{};
};

// Alg. 2 on g; leaves the side bitmap in g->w.best_side (canonical polarity)
int solve_impl(mc_graph *g, const mc_options &o, cudaStream_t s, SolveOut &out) {
    Work &w = g->w;
    const int n0 = g->n0;
    mc_stats &S = out.st;
    memset(&S, 0, sizeof(S));
    S.n_input = n0;
    S.m_input = g->arcs0 / 2;
    Timer total(s);
    PhaseClock ph(g->events, s);
    i64 bytes = 0;
    const long long launches0 = g_launches;
    cudaEvent_t ka, kb;
    cudaEventCreate(&ka);
    cudaEventCreate(&kb);
    struct EvFree {
        cudaEvent_t a, b;
        ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev_free{ka, kb};

    // Components are found only where they matter: a disconnected graph has
    // lambda = 0, which the exact loop reaches by itself (a scan that covers
    // a whole component sees alpha = 0; contraction leaves degree-0
    // vertices); its side is then set to every component but vertex 0's.
    auto component_side = [&](bool *disconnected) -> int {
        int nc = 0;
        MC_TRY(connected_components(g->G0, w, &nc, s));
        *disconnected = nc > 1;
        if (nc > 1) MC_TRY(side_from_component(w, n0, s));
        return MC_OK;
    };
    if (g->delta0 >= (i64)0x7FFFFFFE - 1) {
        bool disc = false;
        MC_TRY(component_side(&disc));
        if (!disc) return MC_EOVERFLOW;
        MC_TRY(side_canon(w, n0, s));
        out.lam = 0;
        S.ms_total = total.ms();
        return MC_OK;
    }

    // lambda-hat = delta with the trivial cut of a minimum-degree vertex
    MC_TRY(iota_i32(w.orig, n0, s));
    i64 lam = g->delta0;
    MC_TRY(side_from_vertex(w, n0, g->argmin0, s));
    bytes += g->G0.arcs * 8 + (i64)n0 * 12;  // degree sweep

    ScanConfig cfg;
    cfg.pq_fifo = o.pq_order == MC_PQ_FIFO;
    cfg.warps = o.scans_per_round;
    cfg.budget = o.region_budget;
    cfg.seed = o.seed;
    cfg.visits = o.visits;
    int rounds = 0, fallbacks = 0;
    const int tail_n = o.tail_vertices == 0 ? 256 : (o.tail_vertices > 4096 ? 4096 : o.tail_vertices);
    const bool verbose = getenv("MC_VERBOSE") != nullptr;

    // Alg. 2's loop from `cur`, contracting into the free buffer of Ga / Gb;
    // lowers lam and records sides through w.orig
    //
    // thr is the bound the round's tests and scans unite at (the value of
    // st->lam on the device): lam itself, or in the approximation mode
    // Matula's min(lam, ceil(approx_milli * delta / 1000)) with delta the
    // minimum degree of the current graph.  A scan whose alpha falls below
    // thr has found a real cut, which lowers lam as well.
    auto exact_loop = [&](DevGraph cur, DevGraph *nxt) -> int {
    int guard = 0;
    i64 delta_cur = g->delta0;
    if (o.approx_milli > 0 && cur.rp != g->G0.rp && cur.n >= 2) {
        MC_TRY(min_degree(cur, w, s));
        MC_TRY(status_read(w, s));
        delta_cur = w.h_st->mindeg;
    }
    auto threshold = [&]() -> i64 {
        if (o.approx_milli <= 0) return lam;
        const i64 a = o.approx_milli;
        i64 t = delta_cur / 1000 * a + (delta_cur % 1000 * a + 999) / 1000;  // ceil(a * delta / 1000)
        if (t < 1) t = 1;
        return t < lam ? t : lam;
    };
    while (cur.n >= 2 && lam > 0) {
        if (++guard > 4 * n0 + 64) return MC_EINTERNAL;
        // a small remainder: its rounds in one single-warp launch
        if (tail_n > 0 && cur.n <= tail_n && cur.arcs <= 64LL * tail_n) {
            long long lt = lam;
            MC_TRY(tail_solve(cur, w, tail_n, &lt, o.seed ^ (u64)rounds, o.pr_level,
                              o.pq_order == MC_PQ_FIFO, n0, s));
            ph.mark(&S.ms_tail);
            if (verbose)
                fprintf(stderr, "[mc] tail n=%d arcs=%lld lam %lld -> %lld (%.3f ms)\n", cur.n,
                        (long long)cur.arcs, (long long)lam, lt, ph.last_ms());
            lam = lt;
            ++S.tail_launches;
            break;
        }
        cfg.round = rounds + guard;
        i64 thr = threshold();
        MC_TRY(round_start(w, cur.n, thr, s));
        // PR1/PR2 and the degree-2 rule on the input graph pass nothing when
        // every weight is below lambda-hat and half of delta and no row has
        // two arcs (unit-weight graphs with delta >= 3): skipped there
        const bool pr12_idle = cur.rp == g->G0.rp && g->wmax0 < thr && 2 * g->wmax0 <= g->delta0 &&
                               g->two_arc_rows0 == 0;
        if (o.pr_level > 0 && !pr12_idle) {
            MC_TRY(pr_tests_budget(cur, w, thr, 1, o.pr_level < 2 ? o.pr_level : 2, 64, s));
            bytes += cur.arcs * 16;
        }
        ph.mark(&S.ms_pr);
        // concurrent capped scans; returns the round's cumulative unions and
        // records a side if some scan's alpha lowered lambda-hat
        auto scan_round = [&](int budget, i64 *unions_out) -> int {
            ScanConfig c2 = cfg;
            c2.budget = budget;
            c2.lam_hint = thr;
            MC_CUDA(cudaEventRecord(ka, s));
            MC_TRY(capforest_parallel(cur, w, c2, s));
            MC_CUDA(cudaEventRecord(kb, s));
            MC_TRY(status_read(w, s));
            float t = 0;
            cudaEventElapsedTime(&t, ka, kb);
            S.ms_scan_kernel += t;
            S.scan_launches += 1;
            const Status st = *w.h_st;
            S.scanned_arcs += st.scanned_arcs;
            S.scanned_verts += st.scanned_verts;
            if (verbose)
                fprintf(stderr, "[mc] round %d n=%d arcs=%lld lam=%lld budget=%d unions=%lld scans=%lld "
                        "scanned_v=%lld scanned_a=%lld black=%lld lam_after=%lld (%.3f ms)\n", rounds,
                        cur.n, (long long)cur.arcs, (long long)lam, budget, (long long)st.unions,
                        (long long)st.scans, (long long)st.scanned_verts, (long long)st.scanned_arcs,
                        (long long)st.blacklisted, (long long)st.lam, t);
            bytes += st.scanned_arcs * 8 + st.scanned_verts * 24;
            if (st.lam < thr && st.best_scan > 0) {
                MC_TRY(side_from_scan(w, n0, st.best_scan, st.best_len, s));
                lam = st.lam;
                thr = st.lam;
            }
            *unions_out = st.unions;
            return MC_OK;
        };
        i64 unions = 0;
        MC_TRY(scan_round(cfg.budget, &unions));
        ph.mark(&S.ms_capforest);
        // a poor round: the triangle tests PR3/PR4 add their unions, on the
        // edges whose shorter row has at most 16 arcs (their work grows with
        // the square of that row: measured on R-MAT 10-cores, 16 arcs beat
        // 24, 32 and 64 end to end, 17.3 against 17.5, 20.7 and 25.0 ms)
        if (o.pr_level >= 3 && unions * 4 < cur.n) {
            MC_TRY(pr_tests_budget(cur, w, thr, 3, o.pr_level, 16, s));
            MC_TRY(status_read(w, s));
            unions = w.h_st->unions;
            bytes += cur.arcs * 16;
            ph.mark(&S.ms_pr);
        }
        // nothing united: wide scans first, then one full scan (Alg. 2); a
        // small graph goes to the full scan at once (measured on two blocks of
        // 2048 vertices: wide scans 0.56 ms for no union, the full scan 1-2 ms)
        if (unions == 0 && !full_scan_is_small(cur.n, thr, cfg.pq_fifo)) {
            MC_TRY(scan_round(1536, &unions));
            ph.mark(&S.ms_capforest);
        }
        if (unions == 0) {
            const i64 thr_before = thr;
            ScanConfig cf = cfg;
            cf.lam_hint = thr;
            MC_TRY(capforest_full(cur, w, cf, s));
            MC_TRY(status_read(w, s));
            const Status st = *w.h_st;
            S.scanned_arcs += st.scanned_arcs;
            S.scanned_verts += st.scanned_verts;
            bytes += st.scanned_arcs * 8 + st.scanned_verts * 24;
            if (st.lam < thr && st.best_scan > 0) {
                MC_TRY(side_from_scan(w, n0, st.best_scan, st.best_len, s));
                lam = st.lam;
                thr = st.lam;
            }
            unions = st.unions;
            ++fallbacks;
            if (verbose)
                fprintf(stderr, "[mc] round %d full scan: unions=%lld lam=%lld\n", rounds,
                        (long long)unions, (long long)lam);
            if (unions == 0) {
                ph.mark(&S.ms_capforest);
                if (thr < thr_before) continue;  // lambda-hat dropped inside the scan: rescan
                set_error_detail("full CAPFOREST scan marked no edge");
                return MC_EINTERNAL;
            }
        }
        ph.mark(&S.ms_capforest);
        // contraction; the orig map and the new minimum degree ride on its
        // final status read
        MC_TRY(contract_graph(cur, *nxt, w, lam, true, 0, s, [&]() -> int {
            MC_TRY(orig_update(w, n0, s));
            return min_degree(*nxt, w, s);
        }));
        if (w.h_st->err & kErrOverflow) return MC_EOVERFLOW;
        if (w.h_st->err & kErrNoProgress) return MC_EINTERNAL;
        bytes += cur.arcs * 20 + w.last_emitted * 12 + (i64)cur.n * 16 + (i64)n0 * 8;
        if (nxt->n >= 2 && w.h_st->mindeg < lam) {
            lam = w.h_st->mindeg;
            MC_TRY(side_from_vertex(w, n0, w.h_st->argmin, s));
        }
        delta_cur = w.h_st->mindeg;
        ph.mark(&S.ms_contract);
        if (verbose)
            fprintf(stderr, "[mc]   contract -> n=%d arcs=%lld emitted=%lld (%.3f ms) lam=%lld\n", nxt->n,
                    (long long)nxt->arcs, (long long)w.last_emitted, ph.last_ms(), (long long)lam);
        cur = *nxt;
        nxt = (nxt == &g->Ga) ? &g->Gb : &g->Ga;
        ++rounds;
    }
    return MC_OK;
    };

    // the label-propagation bound (VieCut, Sec. 2.3 / 3.1.1) on a contracted
    // copy: every candidate is the weight of a real cut of G
    const size_t bound_begin = ph.span_begin();
    Proposer *pp = o.proposer ? reinterpret_cast<Proposer *>(o.proposer) : nullptr;
    if (o.bound == MC_BOUND_LP || o.bound == MC_BOUND_BEST) {
        MC_TRY(lp_bound(g, o, lam, s, verbose, bytes, [&](DevGraph c, DevGraph *nx) { return exact_loop(c, nx); },
                        o.bound == MC_BOUND_BEST ? pp : nullptr));
        MC_TRY(iota_i32(w.orig, n0, s));
    } else if (o.bound == MC_BOUND_LEARNED && pp) {
        // the learned bound on its own: one level of label-propagation
        // clusters (the graph the network was trained on), then the
        // proposer's sweep cut over them; the clusters' own minimum degree is
        // the LP bound's and is not taken here
        int nc = 0;
        MC_TRY(cluster_level0(g, o.lp_iters > 0 ? o.lp_iters : 2, o.seed ^ 0x9E37ULL, lam, &nc, s));
        bytes += (g->G0.arcs * 12 + (i64)n0 * 12) * 2 * (o.lp_iters > 0 ? o.lp_iters : 2) + g->G0.arcs * 20;
        if (nc >= 2) MC_TRY(proposer_on_clusters(g, *pp, g->Ga, w.h_st->mindeg, lam, verbose, s));
        MC_TRY(iota_i32(w.orig, n0, s));
    }
    S.bound_initial = lam;
    ph.span_end(bound_begin, &S.ms_bound);
    const int bound_rounds = rounds;
    rounds = 0;
    MC_TRY(exact_loop(g->G0, &g->Ga));
    (void)bound_rounds;
    if (lam == 0) {
        bool disc = false;
        MC_TRY(component_side(&disc));
    }
    MC_TRY(side_canon(w, n0, s));
    S.rounds = rounds;
    S.fallback_rounds = fallbacks;
    S.bytes_alg = bytes;
    S.kernel_launches = g_launches - launches0;
    out.lam = lam;
    S.ms_total = total.ms();
    ph.finish();
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_options_default(mc_options *opt) {
    if (!opt) return MC_EINVAL;
    memset(opt, 0, sizeof(*opt));
    opt->pq_order = MC_PQ_LIFO;
    opt->bound = MC_BOUND_DEGREE;
    opt->pr_level = 4;
    opt->scans_per_round = 0;
    opt->region_budget = 0;
    opt->lp_iters = 0;
    opt->seed = 0x1234ABCDULL;
    opt->cuda_stream = nullptr;
    return MC_OK;
}

int mc_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                    int32_t flags, mc_graph **out) {
    return create_impl(n, row_ptr, col, w, flags, out);
}

int mc_graph_destroy(mc_graph *g) {
    if (!g) return MC_EINVAL;
    if (!park_shell(g)) destroy_all(g);
    return MC_OK;
}

int mc_graph_size(const mc_graph *g, int64_t *n, int64_t *m) {
    if (!g) return MC_EINVAL;
    if (n) *n = g->n0;
    if (m) *m = g->arcs0 / 2;
    return MC_OK;
}

int mc_min_cut(mc_graph *g, const mc_options *opt, int64_t *lambda_out, uint32_t *side_bitmap,
               mc_stats *stats) {
    if (!g || !lambda_out) return MC_EINVAL;
    mc_options o;
    if (opt) o = *opt; else mc_options_default(&o);
    if (o.pr_level < 0 || o.pr_level > 4 || o.approx_milli < 0 || o.approx_milli > 500 || o.visits < 0 ||
        o.visits > 8)
        return MC_EINVAL;
    cudaStream_t s = pick_stream(g, opt);
    SolveOut so;
    int rc = solve_impl(g, o, s, so);
    if (rc != MC_OK) {
        cudaStreamSynchronize(s);
        return rc;
    }
    *lambda_out = so.lam;
    if (side_bitmap) {
        size_t bytes = sizeof(uint32_t) * (size_t)((g->n0 + 31) / 32);
        MC_CUDA(cudaMemcpyAsync(side_bitmap, g->w.best_side, bytes,
                                g->device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaStreamSynchronize(s));
    if (stats) *stats = so.st;
    return MC_OK;
}

int mc_batch_min_cut(int32_t G, const int64_t *vtx_off, const int64_t *arc_off, const int32_t *row_ptr,
                     const int32_t *col, const int32_t *w, const mc_options *opt, int64_t *lambdas,
                     uint32_t *bitmaps, const int64_t *bitmap_word_off, mc_stats *stats) {
    if (G < 0 || !vtx_off || !arc_off || !row_ptr || !lambdas) return MC_EINVAL;
    if (G > 0 && arc_off[G] > 0 && (!col || !w)) return MC_EINVAL;
    if (bitmaps && !bitmap_word_off) return MC_EINVAL;
    mc_options o;
    if (opt) o = *opt; else mc_options_default(&o);
    const long long l0 = g_launches;
    double ms = 0;
    int rc = batch_solve(G, (const long long *)vtx_off, (const long long *)arc_off, row_ptr, col, w, o,
                         (long long *)lambdas, bitmaps, (const long long *)bitmap_word_off, -1, &ms);
    if (rc != MC_OK) return rc;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_input = G > 0 ? vtx_off[G] : 0;
        stats->m_input = G > 0 ? arc_off[G] / 2 : 0;
        stats->ms_total = ms;
        stats->kernel_launches = g_launches - l0;
    }
    return MC_OK;
}

int mc_batch_autotune(int32_t G, const int64_t *vtx_off, const int64_t *arc_off, const int32_t *row_ptr,
                      const int32_t *col, const int32_t *w, const mc_options *opt, int32_t *best_shape,
                      double *ms_per_shape, int32_t max_shapes) {
    if (G < 1 || !vtx_off || !arc_off || !row_ptr || !col || !w) return MC_EINVAL;
    mc_options o;
    if (opt) o = *opt; else mc_options_default(&o);
    std::vector<long long> lam((size_t)G);
    const int ns = batch_shapes();
    int best = 0;
    double best_ms = 1e300;
    for (int k = 0; k < ns; ++k) {
        double t = 1e300;
        for (int rep = 0; rep < 2; ++rep) {
            double ms = 0;
            MC_TRY(batch_solve(G, (const long long *)vtx_off, (const long long *)arc_off, row_ptr, col, w, o,
                               lam.data(), nullptr, nullptr, k, &ms));
            if (ms < t) t = ms;
        }
        if (ms_per_shape && k < max_shapes) ms_per_shape[k] = t;
        if (t < best_ms) { best_ms = t; best = k; }
    }
    batch_set_shape(best);
    if (best_shape) *best_shape = best;
    return MC_OK;
}

int mc_batch_shape_count(void) { return batch_shapes(); }

int mc_batch_set_shape(int32_t shape) {
    if (shape < -1 || shape >= batch_shapes()) return MC_EINVAL;
    batch_set_shape(shape);
    return MC_OK;
}

int mc_proposer_create(const float *params, uint64_t seed, mc_proposer **out) {
    if (!out) return MC_EINVAL;
    const int P = proposer_nparams();
    std::vector<float> init((size_t)P, 0.f);
    if (params) {
        memcpy(init.data(), params, sizeof(float) * (size_t)P);
    } else {
        // Glorot-uniform weights, zero biases (layout in mc_learn.cu)
        u64 st = seed ^ 0x2545F4914F6CDD1DULL;
        auto uni = [&]() {
            st += 0x9E3779B97F4A7C15ULL;
            u64 z = st;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
            z ^= z >> 31;
            return (double)(z >> 11) * (1.0 / 9007199254740992.0);
        };
        auto fill = [&](int off, int fan_in, int fan_out) {
            const double a = std::sqrt(6.0 / (fan_in + fan_out));
            for (int i = 0; i < fan_in * fan_out; ++i) init[(size_t)off + i] = (float)((2 * uni() - 1) * a);
        };
        fill(0, 8, 64);
        for (int l = 0; l < 3; ++l) fill(8 * 64 + 64 + l * (128 * 64 + 64), 128, 64);
        fill(8 * 64 + 64 + 3 * (128 * 64 + 64), 64, 1);
    }
    Proposer *p = nullptr;
    MC_TRY(proposer_create(&p, init.data()));
    *out = reinterpret_cast<mc_proposer *>(p);
    return MC_OK;
}

int mc_proposer_destroy(mc_proposer *p) {
    if (!p) return MC_EINVAL;
    proposer_destroy(reinterpret_cast<Proposer *>(p));
    return MC_OK;
}

int mc_proposer_get(mc_proposer *p, float *params) {
    if (!p || !params) return MC_EINVAL;
    return proposer_get(reinterpret_cast<Proposer *>(p), params);
}

int mc_proposer_set(mc_proposer *p, const float *params) {
    if (!p || !params) return MC_EINVAL;
    return proposer_set(reinterpret_cast<Proposer *>(p), params);
}

int mc_proposer_forward(mc_proposer *p, mc_graph *g, float *logits) {
    if (!p || !g || !logits) return MC_EINVAL;
    Proposer &pp = *reinterpret_cast<Proposer *>(p);
    MC_TRY(proposer_forward(pp, g->G0, g->delta0, g->stream));
    MC_CUDA(cudaStreamSynchronize(g->stream));
    return proposer_logits_copy(pp, g->n0, logits);
}

static int upload_side(mc_graph *g, const uint32_t *side) {
    MC_CUDA(cudaMemcpyAsync(g->w.best_side, side, sizeof(uint32_t) * (size_t)((g->n0 + 31) / 32),
                            cudaMemcpyHostToDevice, g->stream));
    return MC_OK;
}

int mc_proposer_grad(mc_proposer *p, mc_graph *g, const uint32_t *side, double *loss, float *grad) {
    if (!p || !g || !side || !loss) return MC_EINVAL;
    Proposer &pp = *reinterpret_cast<Proposer *>(p);
    MC_TRY(upload_side(g, side));
    MC_TRY(proposer_forward(pp, g->G0, g->delta0, g->stream));
    MC_TRY(proposer_backward(pp, g->G0, g->w.best_side, loss, g->stream));
    if (grad) MC_TRY(proposer_grad_copy(pp, grad));
    return MC_OK;
}

int mc_proposer_train_step(mc_proposer *p, mc_graph *g, const uint32_t *side, float lr, double *loss) {
    if (!p || !g || !side || !loss || !(lr > 0)) return MC_EINVAL;
    Proposer &pp = *reinterpret_cast<Proposer *>(p);
    MC_TRY(upload_side(g, side));
    MC_TRY(proposer_forward(pp, g->G0, g->delta0, g->stream));
    MC_TRY(proposer_backward(pp, g->G0, g->w.best_side, loss, g->stream));
    MC_TRY(proposer_adam(pp, lr, g->stream));
    MC_CUDA(cudaStreamSynchronize(g->stream));
    return MC_OK;
}

int mc_proposer_bound(mc_proposer *p, mc_graph *g, int64_t *cut, uint32_t *side) {
    if (!p || !g || !cut) return MC_EINVAL;
    Proposer &pp = *reinterpret_cast<Proposer *>(p);
    long long c = 0;
    int k = 0;
    MC_TRY(proposer_forward(pp, g->G0, g->delta0, g->stream));
    MC_TRY(proposer_sweep(pp, g->G0, g->w, &c, &k, g->stream));
    *cut = c;
    if (side) {
        MC_TRY(side_from_rank(g->w, g->n0, k, false, g->stream));
        MC_TRY(side_canon(g->w, g->n0, g->stream));
        MC_CUDA(cudaMemcpyAsync(side, g->w.best_side, sizeof(uint32_t) * (size_t)((g->n0 + 31) / 32),
                                cudaMemcpyDeviceToHost, g->stream));
    }
    MC_CUDA(cudaStreamSynchronize(g->stream));
    return MC_OK;
}

int mc_graph_coarsen(mc_graph *g, int32_t lp_iters, uint64_t seed, mc_graph **out, int32_t *cluster_of) {
    if (!g || !out || lp_iters < 1) return MC_EINVAL;
    *out = nullptr;
    cudaStream_t s = g->stream;
    int nc = 0;
    MC_TRY(cluster_level0(g, lp_iters, seed, g->delta0, &nc, s));
    if (nc < 2) return MC_EINVAL;
    if (cluster_of)
        MC_CUDA(cudaMemcpyAsync(cluster_of, g->w.lab, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    const DevGraph &c = g->Ga;
    std::vector<int> rp((size_t)nc + 1), col((size_t)c.arcs), wt((size_t)c.arcs);
    std::vector<int2> adj((size_t)c.arcs);
    MC_CUDA(cudaMemcpyAsync(rp.data(), c.rp, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost, s));
    if (c.arcs > 0) MC_CUDA(cudaMemcpyAsync(adj.data(), c.adj, sizeof(int2) * adj.size(), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    for (size_t i = 0; i < adj.size(); ++i) {
        col[i] = adj[i].x;
        wt[i] = adj[i].y;
    }
    return create_impl(nc, rp.data(), col.data(), wt.data(), MC_TRUST_INPUT, out);
}

int mc_test_fail_alloc_after(int64_t k) {
    test_fail_alloc_after(k);
    return MC_OK;
}

const char *mc_strerror(int code) {
    static thread_local std::string msg;
    switch (code) {
        case MC_OK: return "ok";
        case MC_EINVAL: return "invalid argument or malformed graph";
        case MC_ENOMEM: return "out of memory";
        case MC_ECUDA: msg = "CUDA error: " + error_detail(); return msg.c_str();
        case MC_ETIMEOUT: return "a bounded device wait timed out";
        case MC_EOVERFLOW: return "weight, degree or bound overflow";
        case MC_EINTERNAL: msg = "internal error: " + error_detail(); return msg.c_str();
        default: return "unknown error";
    }
}

int mc_graph_export(const mc_graph *g, int32_t *row_ptr, int32_t *col, int32_t *w) {
    if (!g) return MC_EINVAL;
    cudaStream_t s = g->stream;
    if (row_ptr)
        MC_CUDA(cudaMemcpyAsync(row_ptr, g->G0.rp, sizeof(int) * ((size_t)g->n0 + 1), cudaMemcpyDeviceToHost, s));
    if ((col || w) && g->arcs0 > 0) {
        std::vector<int2> adj((size_t)g->arcs0);
        MC_CUDA(cudaMemcpyAsync(adj.data(), g->G0.adj, sizeof(int2) * (size_t)g->arcs0, cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        for (i64 i = 0; i < g->arcs0; ++i) {
            if (col) col[i] = adj[(size_t)i].x;
            if (w) w[i] = adj[(size_t)i].y;
        }
    }
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

int mc_step_degrees(mc_graph *g, int64_t *deg) {
    if (!g || !deg) return MC_EINVAL;
    MC_CUDA(cudaMemcpyAsync(deg, g->G0.deg, sizeof(i64) * (size_t)g->n0, cudaMemcpyDeviceToHost, g->stream));
    MC_CUDA(cudaStreamSynchronize(g->stream));
    return MC_OK;
}

int mc_step_contract(mc_graph *g, const int32_t *lab, int32_t nc, int64_t clamp, int32_t *row_ptr,
                     int32_t *col, int32_t *w, int64_t *arcs_out) {
    if (!g || !lab || nc < 1 || nc > g->n0 || !row_ptr || !arcs_out) return MC_EINVAL;
    for (int v = 0; v < g->n0; ++v)
        if (lab[v] < 0 || lab[v] >= nc) return MC_EINVAL;
    cudaStream_t s = g->stream;
    MC_CUDA(cudaMemcpyAsync(g->w.lab, lab, sizeof(int) * (size_t)g->n0, cudaMemcpyHostToDevice, s));
    MC_TRY(round_reset(g->w, 0, s));
    MC_TRY(contract_graph(g->G0, g->Ga, g->w, clamp > 0 ? clamp : LLONG_MAX, false, nc, s));
    MC_TRY(status_read(g->w, s));
    if (g->w.h_st->err & kErrOverflow) return MC_EOVERFLOW;
    *arcs_out = g->Ga.arcs;
    MC_CUDA(cudaMemcpyAsync(row_ptr, g->Ga.rp, sizeof(int) * ((size_t)nc + 1), cudaMemcpyDeviceToHost, s));
    if (g->Ga.arcs > 0 && (col || w)) {
        std::vector<int2> adj((size_t)g->Ga.arcs);
        MC_CUDA(cudaMemcpyAsync(adj.data(), g->Ga.adj, sizeof(int2) * (size_t)g->Ga.arcs, cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        for (i64 i = 0; i < g->Ga.arcs; ++i) {
            if (col) col[i] = adj[(size_t)i].x;
            if (w) w[i] = adj[(size_t)i].y;
        }
    }
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

int mc_step_pr(mc_graph *g, int64_t lam, int32_t level, int32_t *labels) {
    if (!g || !labels || level < 0 || level > 4) return MC_EINVAL;
    cudaStream_t s = g->stream;
    MC_TRY(round_start(g->w, g->n0, lam, s));
    MC_TRY(pr_tests_budget(g->G0, g->w, lam, 1, level, -1, s));
    MC_TRY(flatten_labels(g->w, g->n0, s));
    MC_CUDA(cudaMemcpyAsync(labels, g->w.root, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

int mc_step_capforest(mc_graph *g, int64_t lam, const mc_options *opt, int32_t *labels, int64_t *lam_out,
                      int64_t *unions_out) {
    if (!g || !labels) return MC_EINVAL;
    mc_options o;
    if (opt) o = *opt; else mc_options_default(&o);
    cudaStream_t s = g->stream;
    ScanConfig cfg;
    cfg.pq_fifo = o.pq_order == MC_PQ_FIFO;
    cfg.warps = o.scans_per_round;
    cfg.budget = o.region_budget;
    cfg.seed = o.seed;
    cfg.lam_hint = lam;
    cfg.visits = o.visits;
    MC_TRY(round_start(g->w, g->n0, lam, s));
    MC_TRY(capforest_parallel(g->G0, g->w, cfg, s));
    MC_TRY(flatten_labels(g->w, g->n0, s));
    MC_TRY(status_read(g->w, s));
    MC_CUDA(cudaMemcpyAsync(labels, g->w.root, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (lam_out) *lam_out = g->w.h_st->lam;
    if (unions_out) *unions_out = g->w.h_st->unions;
    return MC_OK;
}

int mc_step_capforest_range(mc_graph *g, int64_t lam, const mc_options *opt, int32_t lo, int32_t hi,
                            int32_t *labels, int64_t *lam_out, int64_t *unions_out, uint32_t *side_bitmap) {
    if (!g || !labels || lo < 0 || hi < lo || hi > g->n0) return MC_EINVAL;
    mc_options o;
    if (opt) o = *opt; else mc_options_default(&o);
    cudaStream_t s = g->stream;
    Work &w = g->w;
    ScanConfig cfg;
    cfg.pq_fifo = o.pq_order == MC_PQ_FIFO;
    cfg.warps = o.scans_per_round;
    cfg.budget = o.region_budget;
    cfg.seed = o.seed;
    cfg.lam_hint = lam;
    cfg.visits = o.visits;
    cfg.lo = lo;
    cfg.hi = hi;
    MC_TRY(round_start(w, g->n0, lam, s));
    MC_TRY(capforest_parallel(g->G0, w, cfg, s));
    MC_TRY(flatten_labels(w, g->n0, s));
    MC_TRY(status_read(w, s));
    const Status st = *w.h_st;
    MC_CUDA(cudaMemcpyAsync(labels, w.root, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    if (side_bitmap) {
        // the prefix of the scan whose alpha lowered the bound (Sec. 3.3),
        // over this graph's vertices; all zero when no scan lowered it
        MC_TRY(iota_i32(w.orig, g->n0, s));
        if (st.lam < lam && st.best_scan > 0) MC_TRY(side_from_scan(w, g->n0, st.best_scan, st.best_len, s));
        else MC_CUDA(cudaMemsetAsync(w.best_side, 0, sizeof(uint32_t) * (size_t)((g->n0 + 31) / 32), s));
        MC_CUDA(cudaMemcpyAsync(side_bitmap, w.best_side, sizeof(uint32_t) * (size_t)((g->n0 + 31) / 32),
                                cudaMemcpyDeviceToHost, s));
    }
    MC_CUDA(cudaStreamSynchronize(s));
    if (lam_out) *lam_out = st.lam;
    if (unions_out) *unions_out = st.unions;
    return MC_OK;
}

int mc_step_capforest_full(mc_graph *g, int64_t lam, int32_t start, int32_t *labels, int64_t *lam_out,
                           int64_t *unions_out) {
    if (!g || !labels || start < 0 || start >= g->n0) return MC_EINVAL;
    cudaStream_t s = g->stream;
    ScanConfig cfg;
    cfg.start = start;
    cfg.lam_hint = lam;
    MC_TRY(round_start(g->w, g->n0, lam, s));
    MC_TRY(capforest_full(g->G0, g->w, cfg, s));
    MC_TRY(flatten_labels(g->w, g->n0, s));
    MC_TRY(status_read(g->w, s));
    MC_CUDA(cudaMemcpyAsync(labels, g->w.root, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (lam_out) *lam_out = g->w.h_st->lam;
    if (unions_out) *unions_out = g->w.h_st->unions;
    return MC_OK;
}

int mc_step_label_prop(mc_graph *g, int32_t iters, uint64_t seed, int32_t *labels) {
    if (!g || !labels || iters < 0) return MC_EINVAL;
    cudaStream_t s = g->stream;
    MC_TRY(label_prop(g->G0, g->w, iters, seed, g->w.lab, s));
    MC_CUDA(cudaMemcpyAsync(labels, g->w.lab, sizeof(int) * (size_t)g->n0, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

}  // extern "C"
