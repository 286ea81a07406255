// mc_internal.cuh -- shared declarations of the libmincut CUDA path.
//
// Device layout of a graph (one GPU, HBM resident):
//   rp   int32[n+1]   CSR row offsets
//   src  int32[arcs]  source vertex of each arc (rows are contiguous, sorted)
//   adj  int2[arcs]   {neighbour, weight} of each arc, rows sorted by neighbour
//   deg  int64[n]     weighted degree (Sec. 2.1)
// Both directions of every undirected edge are stored.  Weights are int32,
// degrees, cut values and lambda-hat are int64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

#include <functional>
#include <string>

#include "mc.h"

namespace mc {

using i64 = long long;
using u64 = unsigned long long;
using u32 = unsigned int;

constexpr int kWarp = 32;
constexpr i64 kInt32Max = 2147483647LL;

// number of kernels launched by this host thread (reported in mc_stats)
extern thread_local long long g_launches;

// ---------------------------------------------------------------- errors --
void set_cuda_error(cudaError_t e, const char *what);
void set_error_detail(const char *msg);

#define MC_CUDA(call)                                         \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) {                              \
            ::mc::set_cuda_error(_e, #call);                  \
            return MC_ECUDA;                                  \
        }                                                     \
    } while (0)

#define MC_TRY(expr)                 \
    do {                             \
        int _rc = (expr);            \
        if (_rc != MC_OK) return _rc; \
    } while (0)

// ------------------------------------------------------------- allocation --
// Device memory comes from the stream-ordered allocator (cudaMallocAsync) on
// the graph's stream; buffers live as long as their owning mc_graph.
int dev_alloc(void **p, size_t bytes, cudaStream_t s);
void test_fail_alloc_after(long long k);  // mc_test_fail_alloc_after
bool test_alloc_hook_armed();               // the hook counts allocations now
void dev_free(void *p, cudaStream_t s);

template <class T>
int dev_alloc_n(T **p, size_t n, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T), s);
}

// ------------------------------------------------------------------ graph --
struct DevGraph {
    int n = 0;
    i64 arcs = 0;
    int *rp = nullptr;
    int *src = nullptr;
    int2 *adj = nullptr;
    i64 *deg = nullptr;
};

// Device-resident status block, read back once per phase.
struct Status {
    i64 lam;            // lambda-hat (atomicMin target)
    i64 unions;         // successful unions this round
    i64 scanned_arcs;   // arcs read by CAPFOREST
    i64 scanned_verts;  // vertices scanned by CAPFOREST
    i64 scans;          // scans started
    i64 blacklisted;    // pops that hit another scan's vertex
    i64 count;          // generic counter (emitted arcs, roots, ...)
    i64 count2;         // second generic counter
    i64 mindeg;         // minimum weighted degree of the current graph
    int argmin;         // smallest vertex with that degree
    int err;            // error bits (kErr*)
    u64 cursor;         // start-vertex cursor of the concurrent scans
    int scan_ids;       // scan id counter
    int best_scan;      // scan whose alpha set lambda-hat (or -1)
    int best_len;       // prefix length of that scan
    int flip;           // the side bitmap's vertex-0 bit, before canonical polarity
    // graph creation: arcs running up and down, and a missing or unequal
    // mirror, seen while the input is built (valid when it is canonical)
    i64 sym_up, sym_down;
    int sym_bad, pad_;
};

constexpr int kErrAsym = 1;       // asymmetric input
constexpr int kErrRange = 2;      // neighbour out of range / bad offsets
constexpr int kErrNegW = 4;       // negative weight
constexpr int kErrOverflow = 8;   // weight or degree overflow
constexpr int kErrNoProgress = 16;

// --------------------------------------------------------------- launches --
int num_sms();

// device-wide exclusive scan of int32 counts into int32 offsets (one launch
// up to 2^19 items, two beyond); *d_total receives the sum (may be nullptr).
// tmp must hold scan_tmp_words(n) ints, cleared whole once by scan_tmp_clear,
// and serve one stream; a stuck wait sets kErrNoProgress in *err.
size_t scan_tmp_words(i64 n);
int scan_tmp_clear(int *tmp, size_t words, cudaStream_t s);
int exclusive_scan_i32(const int *d_in, int *d_out, i64 n, int *d_total, int *tmp, int *err,
                       cudaStream_t s);

// LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
// Buffers A hold the input; the result ends in A or B (returned via *in_b).
// tmp must hold radix_tmp_words(n) uint32.
size_t radix_tmp_words(i64 n);
int radix_sort_pairs(u64 *keysA, int *valsA, u64 *keysB, int *valsB, i64 n, int bits,
                     u32 *tmp, int *scan_tmp, int *err, bool *in_b, cudaStream_t s);

// Contraction workspace.
constexpr int kMinDegBlocks = 1024;  // blocks of one min_degree launch at most
constexpr int kRedMinDone = 2 * kMinDegBlocks;
constexpr int kRedBestDone = 2 * kMinDegBlocks + 1;
constexpr int kRedWords = 2 * kMinDegBlocks + 2;

struct Work {
    // per-vertex (sized n0)
    int *par = nullptr;      // union-find parents
    int *root = nullptr;     // union-find roots after a flatten (labels)
    int *lab = nullptr;      // relabel map
    int *T = nullptr;        // scan owner of each vertex (0 = unvisited)
    int *order = nullptr;    // visit index inside the owning scan
    int *cnt = nullptr;      // per-vertex counts / flags
    int *orig = nullptr;     // original vertex -> current vertex
    int *scan_tmp = nullptr;
    // min_degree's per-block pairs and block counter, the best-scan search's
    // block counter (kRed* below)
    i64 *red = nullptr;
    // per-arc (sized arcs0)
    u64 *keysA = nullptr, *keysB = nullptr;
    int *valsA = nullptr, *valsB = nullptr;
    u32 *radix_tmp = nullptr;
    // per-scan records
    i64 *rec_alpha = nullptr;
    int *rec_len = nullptr;
    // fallback scan state (dense, sized n0 / arcs0)
    int *fb_r = nullptr;
    u32 *fb_pool = nullptr;
    // side bitmap of the best cut so far (original ids)
    u32 *best_side = nullptr;
    // status
    Status *st = nullptr;
    Status *h_st = nullptr;  // pinned mirror
    i64 cap_n = 0, cap_arcs = 0;
    i64 last_emitted = 0;    // arcs emitted by the last contraction
    // single-warp tail solver scratch (allocated on first use)
    unsigned char *tail = nullptr;
    size_t tail_bytes = 0;
    // bucket bitmaps of the block-wide full scan (allocated on first use)
    u32 *blk = nullptr;
    size_t blk_words = 0;
};

int work_alloc(Work &w, i64 n0, i64 arcs0, cudaStream_t s);
void work_free(Work &w, cudaStream_t s);
int graph_alloc(DevGraph &g, i64 n, i64 arcs, cudaStream_t s);
void graph_free(DevGraph &g, cudaStream_t s);

// read the status block back (synchronises the stream)
int status_read(Work &w, cudaStream_t s);

// ---------------------------------------------------------- path steps --
// Sec. 2.1 contraction of `in` by union-find blocks in w.par (roots are the
// smallest member): writes `out`, its degrees, lambda-hat update candidates
// (st->mindeg / st->argmin) and w.lab (old vertex -> new vertex).  Merged
// weights are clamped to `clamp` (> 0).  If `flatten` is false, w.lab holds
// ready labels in [0, nc) with nc given.
// `post` (may be empty) launches more work before the final status read,
// whose Status copy the caller may then use; w.last_emitted = arcs emitted.
int contract_graph(const DevGraph &in, DevGraph &out, Work &w, i64 clamp, bool flatten, int nc,
                   cudaStream_t s, const std::function<int()> &post = {});

// canonicalise raw CSR arrays (device) into `out` (drops self-loops / zero
// weights, sums parallel arcs, sorts rows); checks symmetry if asked.
// Input still arriving from the host, in chunks of whole rows: chunk k holds
// rows [row_split[k], row_split[k + 1]) and is on the device once ready[k]
// has fired; arcs is the input's arc count (known on the host).
struct StagedInput {
    int chunks = 0;
    const int *row_split = nullptr;
    cudaEvent_t *ready = nullptr;
    i64 arcs = 0;
};
int canonicalize(int n, const int *rp, const int *col, const int *w, bool check_sym,
                 DevGraph &out, Work &wk, cudaStream_t s,
                 const StagedInput *staged = nullptr);

int union_find_init(int *par, int n, cudaStream_t s);
int connected_components(const DevGraph &g, Work &w, int *ncomp, cudaStream_t s);

// minimum degree + smallest argmin into st->mindeg / st->argmin
int min_degree(const DevGraph &g, Work &w, cudaStream_t s);
// largest arc weight into st->count, rows with exactly two arcs into st->count2
int graph_stats(const DevGraph &g, Work &w, cudaStream_t s);

// concurrent capped CAPFOREST (Alg. 1): unions into w.par, alpha updates
// into st->lam, owners in w.T / w.order, records in w.rec_*.
struct ScanConfig {
    int pq_fifo = 0;
    int warps = 0;         // concurrent scan warps (0 = auto)
    int budget = 0;        // touched-vertex budget per scan (0 = auto)
    u64 seed = 0;
    int round = 0;
    int start = -1;        // full scan start vertex (-1 = from seed and round)
    long long lam_hint = 0; // lambda-hat at launch (selects the queue kind)
    int visits = 1;        // scans that may scan one vertex (concurrent scans)
    int lo = 0, hi = -1;   // concurrent scans scan only vertices in [lo, hi) (hi < 0: all)
};
int capforest_parallel(const DevGraph &g, Work &w, const ScanConfig &cfg, cudaStream_t s);
// one full CAPFOREST scan (Alg. 3) from a start vertex, single warp
int capforest_full(const DevGraph &g, Work &w, const ScanConfig &cfg, cudaStream_t s);
// true when capforest_full runs the one-warp scan of a small graph (n <= 8192,
// bound <= 63, largest-key order), whose cost is a few wide scans'
bool full_scan_is_small(int n, long long cap, bool fifo);

// side bitmaps (original vertex ids, n0 bits)
int side_from_vertex(Work &w, int n0, int vertex, cudaStream_t s);
int side_from_scan(Work &w, int n0, int scan, int len, cudaStream_t s);
int side_from_component(Work &w, int n0, cudaStream_t s);  // par = CC roots
int orig_update(Work &w, int n0, cudaStream_t s);           // orig = lab[orig]

// tests lo..level; PR3/PR4 only on edges whose shorter row has <= budget arcs
// (every edge if budget < 0)
int pr_tests_budget(const DevGraph &g, Work &w, i64 lam, int lo, int level, int budget,
                    cudaStream_t s);
int flatten_labels(Work &w, int n, cudaStream_t s);   // w.root[v] = root of v in w.par
int round_reset(Work &w, i64 lam, cudaStream_t s);    // st->lam = lam, counters = 0
int round_start(Work &w, int n, i64 lam, cudaStream_t s);  // union_find_init + round_reset
int side_canon(Work &w, int n0, cudaStream_t s);
int iota_i32(int *a, int n, cudaStream_t s);
const std::string &error_detail();

// The full scan on caller-provided state (the allocation-free entry point):
// par = union-find parents (initialised), T and r zeroed, st->lam set, a
// pool of `pool` entries each for eslot / enext, and `blk` (blk_words words)
// for the block-wide scan's bucket bitmaps; unions are applied directly.
// Picks the same kernel as capforest_full for the same graph and bound.
int capforest_full_raw(const DevGraph &g, int *par, int *T, int *order, Status *st, i64 *rec_alpha,
                       int *rec_len, int *r, int *eslot, int *enext, int pool, u32 *blk, size_t blk_words,
                       int start, cudaStream_t s);
// block-wide full scan limits: keys 0..kBlkMaxCap, at most kBlkMaxN
// vertices, whole state on chip up to kBlkOnChipBytes of shared memory
constexpr int kBlkMaxCap = 1023;
constexpr int kBlkMaxN = 1 << 20;
constexpr size_t kBlkOnChipBytes = 200 * 1024;
// words of bucket bitmaps the block-wide full scan needs off chip (0 when its
// state fits on chip)
size_t full_block_words(int n, int cap);
int flatten_raw(int *par, int *root, int *cnt, int n, cudaStream_t s);

// many graphs, one warp per graph (layout of mc_batch_min_cut, host arrays);
// shape < 0 = the tuned or default configuration; *ms_out = kernel time
int batch_solve(int G, const long long *vtx_off, const long long *arc_off, const int *row_ptr,
                const int *col, const int *w, const mc_options &o, long long *lambdas, u32 *bitmaps,
                const long long *bitmap_word_off, int shape, double *ms_out);
int batch_shapes();
// the remaining rounds of Alg. 2 on a small graph g in one single-warp launch
// (PR1/PR2 + degree-2 rule, full capped scan, in-warp contraction per
// round); *lam = min(*lam, lambda(g)), the side recorded through w.orig
int tail_solve(const DevGraph &g, Work &w, int limit, long long *lam, u64 seed, int pr_level, int fifo,
               int n0, cudaStream_t s);
int side_from_bits(Work &w, int n0, const u32 *bits, cudaStream_t s);  // bit v = bits[orig[v]]
void batch_set_shape(int shape);
int batch_get_shape();

// learned proposer (mc_learn.cu)
struct Proposer;
int proposer_create(Proposer **out, const float *init);
void proposer_destroy(Proposer *p);
int proposer_set(Proposer *p, const float *w);
int proposer_get(Proposer *p, float *w);
int proposer_nparams();
int proposer_forward(Proposer &p, const DevGraph &g, long long delta, cudaStream_t s);
int proposer_backward(Proposer &p, const DevGraph &g, const unsigned *bits, double *loss, cudaStream_t s);
int proposer_adam(Proposer &p, float lr, cudaStream_t s);
int proposer_grad_copy(Proposer &p, float *out);
int proposer_logits_copy(Proposer &p, int n, float *out);
int proposer_sweep(Proposer &p, const DevGraph &g, Work &w, long long *cut, int *k_out, cudaStream_t s);
// bit v = w.root[v] < k, or w.root[w.orig[v]] < k with through_orig (ranks
// of the vertices of a contracted graph)
int side_from_rank(Work &w, int n0, int k, bool through_orig, cudaStream_t s);

// label propagation sweeps on g into labels (int32[n]; uses w.cnt, w.T and
// the radix buffers as scratch)
int label_prop(const DevGraph &g, Work &w, int iters, u64 seed, int *labels, cudaStream_t s);
// labels in w.lab (arbitrary vertex ids) -> dense ids in [0, nc) by the order
// of the label values; uses w.root / w.par as scratch
int compact_labels(Work &w, int n, int *nc, cudaStream_t s);

// ---------------------------------------------------------- device bits --
__device__ __forceinline__ u64 splitmix64(u64 x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// Union-find with parents always below their children (link the larger root
// under the smaller), path halving on finds.  Safe under concurrency: only
// roots are linked (by CAS) and halving only shortens paths to ancestors.
__device__ __forceinline__ int uf_find(int *par, int x) {
    volatile int *p = par;
    while (true) {
        int px = p[x];
        if (px == x) return x;
        int gx = p[px];
        if (gx == px) return px;
        p[x] = gx;
        x = gx;
    }
}

// as uf_union; *root = the root of the merged set (its smallest member)
__device__ __forceinline__ bool uf_union_root(int *par, int a, int b, int *root) {
    while (true) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) { *root = a; return false; }
        if (a > b) { int t = a; a = b; b = t; }
        if (atomicCAS(&par[b], b, a) == b) { *root = a; return true; }
    }
}

__device__ __forceinline__ bool uf_union(int *par, int a, int b) {
    while (true) {
        a = uf_find(par, a);
        b = uf_find(par, b);
        if (a == b) return false;
        if (a > b) { int t = a; a = b; b = t; }
        if (atomicCAS(&par[b], b, a) == b) return true;
    }
}

__device__ __forceinline__ i64 ld_volatile_i64(const i64 *p) {
    return *reinterpret_cast<const volatile i64 *>(p);
}

inline int div_up(i64 a, i64 b) { return (int)((a + b - 1) / b); }

}  // namespace mc
