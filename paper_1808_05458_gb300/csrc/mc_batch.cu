// mc_batch.cu -- many independent graphs at once, one warp per graph.
//
// Each warp runs the whole exact loop of Alg. 2 on its graph, entirely in
// its own scratch (shared memory for the scan's r-values and queue when the
// graph is small enough, a per-warp global slice otherwise):
//   canonicalise (merge parallel arcs, drop self-loops and zero weights) ->
//   components (lambda = 0 if disconnected) -> lambda-hat = delta ->
//   rounds of { Padberg-Rinaldi PR1/PR2 + degree-2 tie rule; one full capped
//   CAPFOREST scan (Alg. 3 with the Lemma 1 cap, from a seeded start); in-warp
//   contraction (Sec. 2.1) with the lambda-hat clamp; lambda-hat = min(., delta) }
//   until one vertex is left; the side is kept as in Sec. 3.3.
// The in-warp contraction is a stable counting sort of the arcs by their new
// source block (lanes of one chunk ranked with match_any, so the result is
// deterministic), then a per-row merge of parallel arcs through a marker
// array over the new vertices (first occurrence kept, weights added with the
// clamp), compacted into the next CSR.
// Warps take graphs from a shared queue ordered by size (largest first).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "mc_internal.cuh"
#include "mc_scan.cuh"

namespace mc {

namespace {

constexpr int kBNB = 256;  // queue buckets per warp

template <int SN>
struct WarpSmem {
    int r[SN];
    union {
        struct {
            unsigned short eslot[SN + SN / 2];
            unsigned short enext[SN + SN / 2];
        } q;             // the bucket queue's entry pool
        struct {
            int rp[SN + 1];                // the row offsets, for the dense on-chip scan
            unsigned short par[SN - 2];    // the union-find of a graph of <= SN - 2 vertices
        } s;             // or the round's on-chip arrays
        struct {
            int acc[SN];               // merged weights by target
            unsigned short lab[SN];    // the new labels of the n vertices
        } c;             // or the on-chip contraction's arrays
    } u;
    int head[kBNB];
    int tail[kBNB];
    u32 bits[kBNB / 32];
    int top;
};

// per-warp global scratch, sized for the largest graph of the batch
struct Scratch {
    int *rpA, *rpB, *rpT, *srcA, *srcB, *eslot, *enext;
    int2 *adjA, *adjB, *adjT;
    i64 *deg;
    int *par, *root, *lab, *cnt, *mark, *T, *order, *orig, *rg;
    u32 *best;
    Status *st;
    i64 *rec_alpha;
    int *rec_len;
};

struct Layout {
    int nmax;
    long long amax;
    size_t bytes;  // per warp
    // byte offsets
    size_t rpA, rpB, rpT, srcA, srcB, eslot, enext, adjA, adjB, adjT, deg, par, root, lab, cnt, mark, T, order,
        orig, rg, best, st, rec_alpha, rec_len;
};

static size_t al(size_t x) { return (x + 255) / 256 * 256; }

static Layout make_layout(int nmax, long long amax) {
    Layout L;
    L.nmax = nmax;
    L.amax = amax;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al(bytes); return r; };
    const size_t N1 = (size_t)nmax + 1, A = (size_t)amax + 2;
    L.rpA = take(4 * N1); L.rpB = take(4 * N1); L.rpT = take(4 * N1);
    L.srcA = take(4 * A); L.srcB = take(4 * A);
    L.eslot = take(4 * A); L.enext = take(4 * A);
    L.adjA = take(8 * A); L.adjB = take(8 * A); L.adjT = take(8 * A);
    L.deg = take(8 * N1);
    L.par = take(4 * N1); L.root = take(4 * N1); L.lab = take(4 * N1); L.cnt = take(4 * N1);
    L.mark = take(4 * N1); L.T = take(4 * N1); L.order = take(4 * N1); L.orig = take(4 * N1);
    L.rg = take(4 * N1);
    L.best = take(4 * (N1 / 32 + 2));
    L.st = take(sizeof(Status));
    L.rec_alpha = take(8 * 4);
    L.rec_len = take(4 * 4);
    L.bytes = o;
    return L;
}

__device__ Scratch scratch_of(unsigned char *base, const Layout &L) {
    Scratch S;
    S.rpA = (int *)(base + L.rpA); S.rpB = (int *)(base + L.rpB); S.rpT = (int *)(base + L.rpT);
    S.srcA = (int *)(base + L.srcA); S.srcB = (int *)(base + L.srcB);
    S.eslot = (int *)(base + L.eslot); S.enext = (int *)(base + L.enext);
    S.adjA = (int2 *)(base + L.adjA); S.adjB = (int2 *)(base + L.adjB); S.adjT = (int2 *)(base + L.adjT);
    S.deg = (i64 *)(base + L.deg);
    S.par = (int *)(base + L.par); S.root = (int *)(base + L.root); S.lab = (int *)(base + L.lab);
    S.cnt = (int *)(base + L.cnt); S.mark = (int *)(base + L.mark); S.T = (int *)(base + L.T);
    S.order = (int *)(base + L.order); S.orig = (int *)(base + L.orig); S.rg = (int *)(base + L.rg);
    S.best = (u32 *)(base + L.best);
    S.st = (Status *)(base + L.st);
    S.rec_alpha = (i64 *)(base + L.rec_alpha);
    S.rec_len = (int *)(base + L.rec_len);
    return S;
}

struct BatchIn {
    int G;
    const long long *voff, *aoff;
    const int *rp, *col, *w;
    const int *order;  // graphs, largest first
    long long *lam_out;
    u32 *bits_out;                // may be null
    const long long *bits_off;    // word offsets, may be null
    int *err_out;
    int *next;                    // work counter
    unsigned char *scratch;
    Layout L;
    u64 seed;
    int pr_level;
    int fifo;
};

// ------------------------------------------------------------ warp tools --
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// exclusive scan of cnt[0..n) into out[0..n], out[n] = total; returns total
__device__ int warp_excl_scan(const int *cnt, int *out, int n) {
    const int lane = lane_id();
    int carry = 0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        const int i = i0 + lane;
        const int v = i < n ? cnt[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (i < n) out[i] = carry + inc - v;
        carry += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) out[n] = carry;
    __syncwarp();
    return carry;
}

// weight add with saturation at `clamp`; sets *ovf if a sum passes INT32_MAX
__device__ __forceinline__ void add_clamped(int *p, int w, long long clamp, int *ovf) {
    int old = *p, assumed;
    do {
        assumed = old;
        long long s = (long long)assumed + w;
        if (s > kInt32Max) *ovf = 1;
        int nv = (int)(s > clamp ? clamp : s);
        old = atomicCAS(p, assumed, nv);
    } while (old != assumed);
}

// (minimum degree, smallest vertex with it) over deg[0..n)
__device__ void warp_min_deg(const i64 *deg, int n, long long *md, int *arg) {
    const int lane = lane_id();
    long long best = LLONG_MAX;
    int bi = INT_MAX;
    for (int v = lane; v < n; v += 32) {
        const long long d = deg[v];
        if (d < best) { best = d; bi = v; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    *md = best;
    *arg = bi;
}

// Contract (in_src, in_adj)[0..m) over n vertices by labels lab[] in [0, nc)
// into the CSR (rp, src, adj, deg) with merged weights clamped to `clamp`.
// Uses tmp_rp / tmp_adj for the row-sorted copy and S.cnt / S.mark.
// Returns the arc count of the result.
__device__ long long warp_contract(const int *in_src, const int2 *in_adj, long long m, const int *lab,
                                   int nc, long long clamp, int *tmp_rp, int2 *tmp_adj, int *rp,
                                   int *src, int2 *adj, i64 *deg, int *cnt, int *mark, int *ovf) {
    const int lane = lane_id();
    for (int a = lane; a < nc; a += 32) cnt[a] = 0;
    __syncwarp();
    for (long long i0 = 0; i0 < m; i0 += 32) {
        const long long i = i0 + lane;
        if (i < m) {
            const int a = lab[in_src[i]], b = lab[in_adj[i].x];
            if (a != b) atomicAdd(&cnt[a], 1);
        }
    }
    __syncwarp();
    warp_excl_scan(cnt, tmp_rp, nc);
    // stable scatter: cursor per row in mark[], lanes of a chunk ranked by match_any
    for (int a = lane; a < nc; a += 32) mark[a] = tmp_rp[a];
    __syncwarp();
    for (long long i0 = 0; i0 < m; i0 += 32) {
        const long long i = i0 + lane;
        int a = -1 - lane, b = 0, c = 0;
        if (i < m) {
            a = lab[in_src[i]];
            b = lab[in_adj[i].x];
            c = in_adj[i].y;
            if (a == b) a = -1 - lane;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, a);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = 0;
        if (a >= 0) base = mark[a];
        __syncwarp();
        if (a >= 0) {
            tmp_adj[base + rank] = make_int2(b, c);
            if (rank == 0) mark[a] = base + __popc(peers);
        }
        __syncwarp();
    }
    // merge parallel arcs row by row: first occurrence keeps the arc
    for (int a = lane; a < nc; a += 32) mark[a] = INT_MAX;
    __syncwarp();
    long long out = 0;
    for (int a = 0; a < nc; ++a) {
        const int lo = tmp_rp[a], hi = tmp_rp[a + 1];
        if (lane == 0) rp[a] = (int)out;
        for (int e = lo + lane; e < hi; e += 32) atomicMin(&mark[tmp_adj[e].x], e);
        __syncwarp();
        for (int e = lo + lane; e < hi; e += 32) {
            const int2 x = tmp_adj[e];
            const int rep = mark[x.x];
            if (rep != e) add_clamped(&tmp_adj[rep].y, x.y, clamp, ovf);
        }
        __syncwarp();
        long long dsum = 0;
        for (int e0 = lo; e0 < hi; e0 += 32) {
            const int e = e0 + lane;
            bool keep = false;
            int2 x = make_int2(0, 0);
            if (e < hi) {
                x = tmp_adj[e];
                keep = mark[x.x] == e;
            }
            const unsigned kb = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const long long pos = out + __popc(kb & ((1u << lane) - 1u));
                const int wv = (int)((long long)x.y > clamp ? clamp : (long long)x.y);
                adj[pos] = make_int2(x.x, wv);
                src[pos] = a;
                dsum += wv;
            }
            out += __popc(kb);
        }
        __syncwarp();
        for (int e = lo + lane; e < hi; e += 32) mark[tmp_adj[e].x] = INT_MAX;
        dsum = warp_sum_ll(dsum);
        if (lane == 0) deg[a] = dsum;
        __syncwarp();
    }
    if (lane == 0) rp[nc] = (int)out;
    __syncwarp();
    return out;
}

// Contraction of a graph on chip (n <= SN vertices, nc < n): the steps of
// warp_contract with the per-vertex arrays in shared memory -- 16-bit labels,
// the counts, then cursors, then first positions of the merge (in r), and
// the merged weights -- so that only the arcs travel through global memory.
// The count and scatter passes load four chunks of arcs a lane at a time, the
// merge reads row bounds 32 rows at a time, and a row of at most 32 arcs is
// merged in registers with the next such row's load already in flight.
// Merged weights saturate at `clamp` from the first addition on.
template <int SN>
__device__ long long warp_contract_chip(const int *in_src, const int2 *in_adj, long long m, const int *lab_g,
                                        int n, int nc, long long clamp, int *tmp_rp, int2 *tmp_adj, int *rp,
                                        int *src, int2 *adj, i64 *deg, WarpSmem<SN> &sm, int *ovf) {
    constexpr int kU = 4;
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = lane_id();
    int *mark = sm.r;
    int *acc = sm.u.c.acc;
    unsigned short *lab = sm.u.c.lab;
    for (int v = lane; v < n; v += 32) lab[v] = (unsigned short)lab_g[v];
    for (int a = lane; a <= nc; a += 32) mark[a] = 0;
    __syncwarp();
    for (long long i0 = 0; i0 < m; i0 += 32 * kU) {
        int s[kU], t[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            const long long i = i0 + 32 * j + lane;
            s[j] = t[j] = 0;
            if (i < m) {
                s[j] = in_src[i];
                t[j] = in_adj[i].x;
            }
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            const int a = lab[s[j]], b = lab[t[j]];
            if (i0 + 32 * j + lane < m && a != b) atomicAdd(&mark[a], 1);
        }
    }
    __syncwarp();
    warp_excl_scan(mark, mark, nc);  // in place: each entry is read and written by its own lane
    for (int a = lane; a <= nc; a += 32) tmp_rp[a] = mark[a];
    __syncwarp();
    // stable scatter: the lanes of a chunk meeting the same row ranked by match_any
    for (long long i0 = 0; i0 < m; i0 += 32 * kU) {
        int s[kU];
        int2 e[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            const long long i = i0 + 32 * j + lane;
            s[j] = 0;
            e[j] = make_int2(0, 0);
            if (i < m) {
                s[j] = in_src[i];
                e[j] = in_adj[i];
            }
        }
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            int a = -1 - lane, b = 0;
            if (i0 + 32 * j + lane < m) {
                a = lab[s[j]];
                b = lab[e[j].x];
                if (a == b) a = -1 - lane;
            }
            const unsigned peers = __match_any_sync(kAll, a);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            int base = 0;
            if (a >= 0) base = mark[a];
            __syncwarp();
            if (a >= 0) {
                tmp_adj[base + rank] = make_int2(b, e[j].y);
                if (rank == 0) mark[a] = base + __popc(peers);
            }
            __syncwarp();
        }
    }
    // merge parallel arcs row by row: the first occurrence keeps the arc
    for (int a = lane; a < nc; a += 32) mark[a] = INT_MAX;
    __syncwarp();
    long long out = 0;
    for (int a0 = 0; a0 < nc; a0 += 32) {
        const int rows = nc - a0 < 32 ? nc - a0 : 32;
        const int bl = lane <= rows ? tmp_rp[a0 + lane] : 0;       // bounds of rows a0 .. a0 + 31
        const int bend = rows == 32 ? tmp_rp[a0 + 32] : 0;         // the end of row a0 + 31
        int lo = __shfl_sync(kAll, bl, 0), hi = __shfl_sync(kAll, bl, 1);
        int2 xn = make_int2(0, 0);
        if (hi - lo <= 32 && lane < hi - lo) xn = tmp_adj[lo + lane];
        for (int k = 0; k < rows; ++k) {
            const int a = a0 + k;
            const int2 x = xn;
            // the next row's bounds, and its arcs if it is short
            const int nhi_l = __shfl_sync(kAll, bl, (k + 2) & 31);
            const int nlo = hi, nhi = k + 2 <= 31 ? nhi_l : (k + 2 == 32 ? bend : nlo);
            if (k + 1 < rows && nhi - nlo <= 32 && lane < nhi - nlo) xn = tmp_adj[nlo + lane];
            if (lane == 0) rp[a] = (int)out;
            long long dsum;
            if (hi - lo <= 32) {
                const bool v = lane < hi - lo;
                if (v) {
                    atomicMin(&mark[x.x], lane);
                    acc[x.x] = 0;
                }
                __syncwarp();
                if (v) add_clamped(&acc[x.x], x.y, clamp, ovf);
                __syncwarp();
                const bool keep = v && mark[x.x] == lane;
                const int wv = keep ? acc[x.x] : 0;
                const unsigned kb = __ballot_sync(kAll, keep);
                if (keep) {
                    const long long pos = out + __popc(kb & ((1u << lane) - 1u));
                    adj[pos] = make_int2(x.x, wv);
                    src[pos] = a;
                }
                out += __popc(kb);
                // weights below 2^31: the two 16-bit halves sum without carry-out
                dsum = (long long)__reduce_add_sync(kAll, (unsigned)wv >> 16) * 65536 +
                       (long long)__reduce_add_sync(kAll, (unsigned)wv & 0xFFFFu);
                __syncwarp();
                if (v) mark[x.x] = INT_MAX;
            } else {
                for (int e = lo + lane; e < hi; e += 32) {
                    const int2 y = tmp_adj[e];
                    atomicMin(&mark[y.x], e);
                    acc[y.x] = 0;
                }
                __syncwarp();
                for (int e = lo + lane; e < hi; e += 32) {
                    const int2 y = tmp_adj[e];
                    add_clamped(&acc[y.x], y.y, clamp, ovf);
                }
                __syncwarp();
                long long ds = 0;
                for (int e0 = lo; e0 < hi; e0 += 32) {
                    const int e = e0 + lane;
                    bool keep = false;
                    int2 y = make_int2(0, 0);
                    if (e < hi) {
                        y = tmp_adj[e];
                        keep = mark[y.x] == e;
                    }
                    const int wv = keep ? acc[y.x] : 0;
                    const unsigned kb = __ballot_sync(kAll, keep);
                    if (keep) {
                        const long long pos = out + __popc(kb & ((1u << lane) - 1u));
                        adj[pos] = make_int2(y.x, wv);
                        src[pos] = a;
                    }
                    out += __popc(kb);
                    ds += wv;
                }
                dsum = warp_sum_ll(ds);
                __syncwarp();
                for (int e = lo + lane; e < hi; e += 32) mark[tmp_adj[e].x] = INT_MAX;
            }
            if (lane == 0) deg[a] = dsum;
            __syncwarp();
            lo = nlo;
            hi = nhi;
            if (k + 1 < rows && (hi - lo > 32)) xn = make_int2(0, 0);
        }
    }
    if (lane == 0) rp[nc] = (int)out;
    __syncwarp();
    return out;
}

// Stable transpose of the arcs (src[i] -> adj[i].x, weight adj[i].y), i in
// [0, m), over n vertices: row v of the result lists (u, c) for every arc
// u -> v in the input's index order; out_src[j] = v.  An input whose arcs
// are ordered by source yields rows sorted by source.
__device__ void warp_transpose(const int *src, const int2 *adj, long long m, int n, int *out_rp,
                               int *out_src, int2 *out_adj, int *cnt, int *cursor) {
    const int lane = lane_id();
    for (int v = lane; v < n; v += 32) cnt[v] = 0;
    __syncwarp();
    for (long long i = lane; i < m; i += 32) atomicAdd(&cnt[adj[i].x], 1);
    __syncwarp();
    warp_excl_scan(cnt, out_rp, n);
    for (int v = lane; v < n; v += 32) cursor[v] = out_rp[v];
    __syncwarp();
    for (long long i0 = 0; i0 < m; i0 += 32) {
        const long long i = i0 + lane;
        int v = -1 - lane, u = 0, c = 0;
        if (i < m) {
            v = adj[i].x;
            c = adj[i].y;
            u = src[i];
        }
        const unsigned peers = __match_any_sync(0xffffffffu, v);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        int base = 0;
        if (v >= 0) base = cursor[v];
        __syncwarp();
        if (v >= 0) {
            out_adj[base + rank] = make_int2(u, c);
            out_src[base + rank] = v;
            if (rank == 0) cursor[v] = base + __popc(peers);
        }
        __syncwarp();
    }
}

// Symmetry of a canonical CSR (every row free of duplicates, arcs ordered by
// source): G is symmetric (every arc (u, v, c) has its mirror (v, u, c))
// exactly when every upward arc finds its mirror and as many arcs run down as
// up (the mirror map is then a bijection).  With rows sorted by neighbour (an
// input with sorted rows keeps them through the merge) a binary search in the
// neighbour's row finds the mirror.  Otherwise: T1 = transpose(G) has rows
// sorted by source, T2 = transpose(T1) is G with its rows sorted, and G is
// symmetric exactly when T1 and T2 are equal entry for entry.
__device__ bool warp_symmetric(const int *rp, const int *src, const int2 *adj, long long m, int n, int *rp1,
                               int *src1, int2 *adj1, int *rp2, int *src2, int2 *adj2, int *cnt, int *cursor) {
    const int lane = lane_id();
    bool unsorted = false;
    for (long long i = lane; i + 1 < m; i += 32)
        unsorted |= src[i] == src[i + 1] && adj[i].x >= adj[i + 1].x;
    if (!__any_sync(0xffffffffu, unsorted)) {
        bool bad = false;
        long long up = 0, down = 0;
        for (long long i = lane; i < m; i += 32) {
            const int u = src[i];
            const int2 e = adj[i];
            if (u < e.x) {
                ++up;
                int lo = rp[e.x], hi = rp[e.x + 1] - 1, found = -1;
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    const int x = adj[mid].x;
                    if (x == u) { found = adj[mid].y; break; }
                    if (x < u) lo = mid + 1; else hi = mid - 1;
                }
                bad |= found != e.y;
            } else {
                ++down;
            }
        }
        return !__any_sync(0xffffffffu, bad) && warp_sum_ll(up) == warp_sum_ll(down);
    }
    warp_transpose(src, adj, m, n, rp1, src1, adj1, cnt, cursor);
    warp_transpose(src1, adj1, m, n, rp2, src2, adj2, cnt, cursor);
    bool bad = false;
    for (int v = lane; v <= n; v += 32) bad |= rp1[v] != rp2[v];
    for (long long i = lane; i < m; i += 32) {
        const int2 a = adj1[i], b = adj2[i];
        bad |= a.x != b.x || a.y != b.y;
    }
    return !__any_sync(0xffffffffu, bad);
}

// flatten the union-find par[0..n) into root[] and number the blocks in
// lab[] (order of the smallest member); returns the block count
// Union-find over 32-bit parents in global memory or 16-bit parents on chip
// (graphs of at most 65535 vertices): the parent of a vertex is always below
// it, a union links the larger root under the smaller by CAS, and a find
// halves the path it walks (only ever shortening paths to ancestors).
template <class P>
__device__ __forceinline__ int wuf_find(P *par, int x) {
    volatile P *p = par;
    while (true) {
        const int px = p[x];
        if (px == x) return x;
        const int gx = p[px];
        if (gx == px) return px;
        p[x] = (P)gx;
        x = gx;
    }
}

template <class P>
__device__ __forceinline__ bool wuf_union(P *par, int a, int b) {
    while (true) {
        a = wuf_find(par, a);
        b = wuf_find(par, b);
        if (a == b) return false;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if ((int)atomicCAS(&par[b], (P)b, (P)a) == b) return true;
    }
}

// the unions a scan recorded (joinx[y] = the vertex whose pop made y join,
// -1 if none), applied after the scan; 16-bit parents when par16 is set
__device__ __forceinline__ void apply_joins(const int *joinx, int n, int *par32, unsigned short *par16,
                                            Counters &cnt) {
    const int lane = lane_id();
    __syncwarp();
    for (int y = lane; y < n; y += 32) {
        const int x = joinx[y];
        if (x >= 0 && (par16 ? wuf_union(par16, x, y) : wuf_union(par32, x, y))) cnt.unions++;
    }
    __syncwarp();
}

template <class P>
__device__ int warp_relabel(P *par, int *root, int *lab, int *cnt, int n) {
    const int lane = lane_id();
    for (int v = lane; v < n; v += 32) {
        const int r = wuf_find(par, v);
        root[v] = r;
        cnt[v] = r == v;
    }
    __syncwarp();
    const int nc = warp_excl_scan(cnt, lab, n);
    for (int v = lane; v < n; v += 32) {
        const int r = root[v];
        if (r != v) lab[v] = lab[r];
    }
    __syncwarp();
    return nc;
}

template <class F>
__device__ void warp_side_bits(u32 *bits, int n0, F f) {
    const int lane = lane_id();
    for (int v0 = 0; v0 < n0; v0 += 32) {
        const int v = v0 + lane;
        const bool b = v < n0 && f(v);
        const unsigned m = __ballot_sync(0xffffffffu, b);
        if (lane == 0) bits[v0 / 32] = m;
    }
    __syncwarp();
}

// One full capped CAPFOREST scan (Alg. 3) of a graph of at most 256
// vertices with a cap C <= 63, r on chip: one bitmap per key over the
// vertices (8 words, in the list queue's head/tail arrays), a pop takes the
// smallest vertex of the largest key.  A queue entry packs into one word,
// (key + 1) << 8 | (255 - vertex), so the next pop is the larger of the
// candidate searched before the popped row is applied and the row's largest
// move (keys only rise): one warp reduction per 32 arcs, no second search.
// Measured on the tail of RHG 2^20 (71 vertices): the list-queue scan took
// about 2000 cycles per pop.
// Joins are recorded in joinx and applied after the scan (apply_joins).
template <int SN>
__device__ void warp_scan_bits(const ScanArgs &A, WarpSmem<SN> &sm, int n, int C, int start, int *joinx,
                               unsigned short *par16, Counters &cnt) {
    static_assert(2 * kBNB >= 64 * 8, "bitmaps of 64 keys fit the head and tail arrays");
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = lane_id();
    u32 *b0 = reinterpret_cast<u32 *>(sm.head);  // (C + 1) x 8 words
    int *r = sm.r;
    for (int i = lane; i < (C + 1) * 8; i += 32) b0[i] = 0;
    for (int v = lane; v < n; v += 32) joinx[v] = -1;
    __syncwarp();
    if (lane == 0) b0[start >> 5] = 1u << (start & 31);  // key 0
    __syncwarp();
    int top = 0;  // keys above top are empty
    auto search = [&]() -> unsigned {
        for (; top >= 0; --top) {
            const u32 w = lane < 8 ? b0[top * 8 + lane] : 0u;
            const unsigned v = __reduce_min_sync(kAll, w ? (unsigned)(lane * 32 + __ffs(w) - 1) : kAll);
            if (v != kAll) return ((unsigned)(top + 1) << 8) | (255u - v);
        }
        top = 0;
        return 0u;
    };
    long long L = ld_volatile_i64(&A.st->lam);
    int Lj = L <= C ? (int)L : INT_MAX;  // the join threshold: none above C
    long long alpha = 0, best = LLONG_MAX;
    int nS = 0, best_len = 0;
    bool alpha_ok = true;
    cnt.scans++;
    unsigned pe = search();
    while (pe != 0u && nS < n) {
        const int p = 255 - (int)(pe & 255u), Kp = (int)(pe >> 8) - 1;
        const int a0 = A.g.rp[p], a1 = A.g.rp[p + 1];
        const int rx = r[p];
        const long long dx = A.g.deg[p];
        if (lane == 0) {
            b0[Kp * 8 + (p >> 5)] &= ~(1u << (p & 31));
            r[p] = kDone;
            A.T[p] = 1;
            A.order[p] = nS;
        }
        __syncwarp();
        ++nS;
        if (rx >= kSat) alpha_ok = false;
        alpha += dx - 2LL * rx;
        if (alpha_ok && nS < n && alpha < L) {
            if (lane == 0) atomicMin(&A.st->lam, alpha);
            best = alpha;
            best_len = nS;
            L = alpha;
            Lj = L <= C ? (int)L : INT_MAX;
        }
        cnt.verts++;
        cnt.arcs += a1 - a0;
        const unsigned qe = search();  // before p's moves change the bitmaps
        __syncwarp();
        unsigned be = qe;
        for (int i0 = a0; i0 < a1; i0 += 32) {
            const int i = i0 + lane;
            const int2 e = i < a1 ? A.g.adj[i] : make_int2(0, 0);
            const int y = e.x;
            unsigned me = 0u;
            if (i < a1) {
                const int ro = r[y];
                if (ro != kDone) {
                    const int rn = sat_add(ro, e.y);
                    r[y] = rn;
                    // a certificate min(r, C) only vouches for bounds <= C
                    if (ro < Lj && Lj <= rn) joinx[y] = p;
                    const int ko = ro == 0 ? -1 : (ro < C ? ro : C), kn = rn < C ? rn : C;
                    if (ko != kn) {
                        const u32 bit = 1u << (y & 31);
                        if (ko >= 0) atomicAnd(&b0[ko * 8 + (y >> 5)], ~bit);
                        atomicOr(&b0[kn * 8 + (y >> 5)], bit);
                        me = ((unsigned)(kn + 1) << 8) | (unsigned)(255 - y);
                    }
                }
            }
            me = __reduce_max_sync(kAll, me);
            be = me > be ? me : be;
        }
        const int kb = (int)(be >> 8) - 1;
        top = kb > top ? kb : top;
        pe = be;
        __syncwarp();
    }
    if (lane == 0) {
        A.rec_alpha[1] = best;
        A.rec_len[1] = best_len;
    }
    apply_joins(joinx, n, A.par, par16, cnt);
}

// One full capped CAPFOREST scan (Alg. 3) of a graph held on chip (n <= SN
// vertices, cap C < 2^25) with no queue beyond the r array itself: the
// vertices fall into 32 groups of B consecutive ones (B a power of two,
// B <= 64), and gmax[g] holds group g's largest key packed with its index,
// (min(r, C) + 1) << 5 | (31 - g), 0 for a group with no reached vertex.  A
// pop is two warp reductions: the best group, then the best vertex in it
// (the smallest vertex of the largest key, as the other queues pop); the
// same loads give the group's maximum without the popped vertex, and every
// key rise is one shared atomicMax on its group's entry.  The row offsets
// are staged on chip in the bucket queue's pool, which this scan leaves
// unused, so a pop's only global round trip is its row's arcs.  A join
// (r crossing the bound) only records its popped vertex in joinx[y] (a
// vertex joins at most once a scan, as r only rises); the unions follow the
// scan in one lane-parallel pass, off the pops' chain of latencies.
template <int SN>
__device__ void warp_scan_dense(const ScanArgs &A, WarpSmem<SN> &sm, int n, int C, int start, int *joinx,
                                unsigned short *par16, Counters &cnt) {
    static_assert(SN <= 2048, "32 groups of at most 64 vertices");
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = lane_id();
    int lgB = 0;
    while ((32 << lgB) < n) ++lgB;
    const int B = 1 << lgB;
    int *r = sm.r;
    int *rps = sm.u.s.rp;
    u32 *gmax = reinterpret_cast<u32 *>(sm.head);
    for (int v = lane; v <= n; v += 32) {
        rps[v] = A.g.rp[v];
        if (v < n) joinx[v] = -1;
    }
    gmax[lane] = 0u;
    __syncwarp();
    long long L = ld_volatile_i64(&A.st->lam);
    int Lj = L <= C ? (int)L : INT_MAX;  // the join threshold: none above C
    long long alpha = 0, best = LLONG_MAX;
    int nS = 0, best_len = 0;
    bool alpha_ok = true;
    cnt.scans++;
    // the vertices popped next, in order: one, or up to kCap at the cap
    constexpr int kCap = 4;
    int nb = 1;
    int bx[kCap] = {start, 0, 0, 0};
    while (nb > 0) {
        // every row of the batch starts its loads before the first pop
        int a0[kCap], a1[kCap];
        long long dxs[kCap];
        int2 e0[kCap];
#pragma unroll
        for (int t = 0; t < kCap; ++t) {
            a0[t] = a1[t] = 0;
            dxs[t] = 0;
            e0[t] = make_int2(0, 0);
            if (t < nb) {
                a0[t] = rps[bx[t]];
                a1[t] = rps[bx[t] + 1];
                dxs[t] = A.g.deg[bx[t]];
                if (lane < a1[t] - a0[t]) e0[t] = A.g.adj[a0[t] + lane];
            }
        }
#pragma unroll
        for (int t = 0; t < kCap; ++t) {
            if (t >= nb) break;
            const int p = bx[t];
            const int rx = r[p];
            __syncwarp();
            if (lane == 0) {
                r[p] = kDone;
                A.T[p] = 1;
                A.order[p] = nS;
            }
            ++nS;
            if (rx >= kSat) alpha_ok = false;
            alpha += dxs[t] - 2LL * rx;
            if (alpha_ok && nS < n && alpha < L) {
                if (lane == 0) atomicMin(&A.st->lam, alpha);
                best = alpha;
                best_len = nS;
                L = alpha;
                Lj = L <= C ? (int)L : INT_MAX;
            }
            cnt.verts++;
            cnt.arcs += a1[t] - a0[t];
            __syncwarp();
            for (int i0 = a0[t]; i0 < a1[t]; i0 += 32) {
                const int i = i0 + lane;
                if (i < a1[t]) {
                    const int2 e = i0 == a0[t] ? e0[t] : A.g.adj[i];
                    const int y = e.x;
                    const int ro = r[y];
                    if (ro != kDone) {
                        const int rn = sat_add(ro, e.y);
                        r[y] = rn;
                        // a certificate min(r, C) only vouches for bounds <= C
                        if (ro < Lj && Lj <= rn) joinx[y] = p;
                        const int ko = ro == 0 ? 0 : (ro < C ? ro : C) + 1, kn = (rn < C ? rn : C) + 1;
                        if (ko != kn) atomicMax(&gmax[y >> lgB], ((u32)kn << 5) | (u32)(31 - (y >> lgB)));
                    }
                }
            }
            __syncwarp();
        }
        if (nS >= n) break;
        // the next pop: best group, then its best vertex
        const u32 top = __reduce_max_sync(kAll, gmax[lane]);
        if (top == 0u) break;
        const int g = 31 - (int)(top & 31u);
        const int v0 = (g << lgB) + lane, v1 = v0 + 32;
        u32 k0 = 0u, k1 = 0u;
        if (lane < B && v0 < n) {
            const int rv = r[v0];
            if (rv != kDone && rv > 0) k0 = ((u32)((rv < C ? rv : C) + 1) << 6) | (u32)(63 - lane);
        }
        if (lane + 32 < B && v1 < n) {
            const int rv = r[v1];
            if (rv != kDone && rv > 0) k1 = ((u32)((rv < C ? rv : C) + 1) << 6) | (u32)(31 - lane);
        }
        const u32 m = __reduce_max_sync(kAll, k0 > k1 ? k0 : k1);
        if (m == 0u) break;  // a group entry always has a reached member
        u32 x0, x1;
        const u32 capk = (u32)C + 1u;
        if ((m >> 6) == capk) {
            // members at the cap go up to kCap at a time, smallest first: no
            // key passes the cap, so each is still a largest key at its pop
            // (a later one's r takes the earlier rows' weights as it would
            // one pop at a time)
            const unsigned s0 = __ballot_sync(kAll, (k0 >> 6) == capk), s1 = __ballot_sync(kAll, (k1 >> 6) == capk);
            unsigned t0 = s0, t1 = s1;
            nb = 0;
#pragma unroll
            for (int t = 0; t < kCap; ++t) {
                if (t0) {
                    bx[t] = (g << lgB) + __ffs(t0) - 1;
                    t0 &= t0 - 1u;
                    nb = t + 1;
                } else if (t1) {
                    bx[t] = (g << lgB) + 32 + __ffs(t1) - 1;
                    t1 &= t1 - 1u;
                    nb = t + 1;
                }
            }
            x0 = (((s0 & ~t0) >> lane) & 1u) ? 0u : k0;
            x1 = (((s1 & ~t1) >> lane) & 1u) ? 0u : k1;
        } else {
            nb = 1;
            bx[0] = (g << lgB) + 63 - (int)(m & 63u);
            x0 = k0 == m ? 0u : k0;
            x1 = k1 == m ? 0u : k1;
        }
        const u32 m2 = __reduce_max_sync(kAll, x0 > x1 ? x0 : x1);
        __syncwarp();
        if (lane == 0) gmax[g] = m2 ? ((m2 >> 6) << 5) | (u32)(31 - g) : 0u;
        __syncwarp();
    }
    if (lane == 0) {
        A.rec_alpha[1] = best;
        A.rec_len[1] = best_len;
    }
    apply_joins(joinx, n, A.par, par16, cnt);
}

// A round whose scan takes the bitmap or the dense queue (graph on chip, cap
// below 2^25, no FIFO order) keeps its union-find on chip, in 16-bit parents
// beside the staged row offsets; other rounds keep it in global memory.
template <int SN>
__device__ __forceinline__ bool round_on_chip(int n, long long lam, int fifo) {
    return n <= SN - 2 && !fifo && lam < (1 << 25);
}

// one full capped CAPFOREST scan of the current graph (Alg. 3); par16 (only
// with round_on_chip) holds the union-find instead of A.par
template <int SN>
__device__ void warp_full_scan(const ScanArgs &A, WarpSmem<SN> &sm, Scratch &S, int n, long long arcs,
                               long long lam, int start, int fifo, unsigned short *par16, Counters &cnt) {
    const int lane = lane_id();
    const bool in_smem = n <= SN;
    int *r = in_smem ? sm.r : S.rg;
    for (int v = lane; v < n; v += 32) { r[v] = 0; S.T[v] = 0; }
    for (int b = lane; b < kBNB; b += 32) { sm.head[b] = -1; sm.tail[b] = -1; }
    if (lane < kBNB / 32) sm.bits[lane] = 0;
    if (lane == 0) {
        sm.top = 0;
        S.st->lam = lam;
        S.st->scan_ids = 1;
    }
    __syncwarp();
    const int C = (int)(lam < (long long)0x7FFFFFFD ? lam : (long long)0x7FFFFFFD);
    if (in_smem && n <= 256 && C <= 63 && !fifo) {
        warp_scan_bits<SN>(A, sm, n, C, start, S.rg, par16, cnt);
    } else if (in_smem && !fifo && C < (1 << 25)) {
        warp_scan_dense<SN>(A, sm, n, C, start, S.rg, par16, cnt);
    } else if (in_smem) {
        BucketQ<unsigned short, kBNB> q;
        q.head = sm.head; q.tail = sm.tail; q.bits = sm.bits; q.eslot = sm.u.q.eslot; q.enext = sm.u.q.enext;
        q.top = &sm.top; q.cap = SN + SN / 2; q.C = C; q.coarse = C + 1 > kBNB; q.fifo = fifo != 0;
        DenseTable tab{r, n};
        scan_one<DenseTable, BucketQ<unsigned short, kBNB>, false, true>(A, tab, q, start, 1, cnt);
    } else {
        BucketQ<int, kBNB> q;
        q.head = sm.head; q.tail = sm.tail; q.bits = sm.bits; q.eslot = S.eslot; q.enext = S.enext;
        q.top = &sm.top; q.cap = (int)(arcs + 2); q.C = C; q.coarse = C + 1 > kBNB; q.fifo = fifo != 0;
        DenseTable tab{r, 0};
        scan_one<DenseTable, BucketQ<int, kBNB>, false, true>(A, tab, q, start, 1, cnt);
    }
    __syncwarp();
}

// Padberg-Rinaldi PR1/PR2 (Sec. 2.2) and the degree-2 tie rule on the graph
// (rp, src, adj, deg) against lambda-hat `lam`: the unions go into par; kPU
// arcs or vertices a lane at a time, so that their loads overlap.  Returns
// this lane's count of successful unions.
template <class P>
__device__ long long pr_unions(P *par, const int *rpA, const int *srcA, const int2 *adjA, const i64 *deg, int n,
                               long long arcs, long long lam, int pr_level) {
    const int lane = lane_id();
    long long un = 0;
    constexpr int kPU = 4;
    for (long long i0 = 0; i0 < arcs; i0 += 32 * kPU) {
        int uu[kPU];
        int2 ee[kPU];
        long long du[kPU], dv[kPU];
#pragma unroll
        for (int j = 0; j < kPU; ++j) {
            const long long i = i0 + 32 * j + lane;
            uu[j] = -1;
            ee[j] = make_int2(-1, 0);
            if (i < arcs) {
                uu[j] = srcA[i];
                ee[j] = adjA[i];
            }
        }
#pragma unroll
        for (int j = 0; j < kPU; ++j) {
            du[j] = dv[j] = 0;
            if (pr_level >= 2 && uu[j] >= 0 && uu[j] < ee[j].x && ee[j].y < lam) {
                du[j] = deg[uu[j]];
                dv[j] = deg[ee[j].x];
            }
        }
#pragma unroll
        for (int j = 0; j < kPU; ++j) {
            if (uu[j] < 0 || uu[j] >= ee[j].x) continue;
            const long long c = ee[j].y;
            const bool ok = c >= lam || (pr_level >= 2 && 2 * c > (du[j] < dv[j] ? du[j] : dv[j]));
            if (ok && wuf_union(par, uu[j], ee[j].x)) ++un;
        }
    }
    if (pr_level >= 2) {
        for (int u0 = 0; u0 < n; u0 += 32 * kPU) {
            int a[kPU], d[kPU];
            int2 f0[kPU], f1[kPU];
#pragma unroll
            for (int j = 0; j < kPU; ++j) {
                const int u = u0 + 32 * j + lane;
                a[j] = d[j] = 0;
                if (u < n) {
                    a[j] = rpA[u];
                    d[j] = rpA[u + 1] - a[j];
                }
            }
#pragma unroll
            for (int j = 0; j < kPU; ++j) {
                f0[j] = f1[j] = make_int2(0, 0);
                if (d[j] == 2) {
                    f0[j] = adjA[a[j]];
                    f1[j] = adjA[a[j] + 1];
                }
            }
#pragma unroll
            for (int j = 0; j < kPU; ++j) {
                const int u = u0 + 32 * j + lane;
                if (d[j] == 2 && f0[j].y == f1[j].y &&
                    wuf_union(par, u, f0[j].x < f1[j].x ? f0[j].x : f1[j].x))
                    ++un;
            }
        }
    }
    __syncwarp();
    return un;
}

// Alg. 2's rounds on the graph in the A buffers of S (n vertices, `arcs`
// arcs, degrees in S.deg): PR1/PR2 + degree-2 rule, one full capped scan,
// in-warp contraction, lambda-hat = min(., delta), until one vertex is left.
// `lam` enters as lambda-hat and leaves as the minimum found; every lowering
// rewrites the side bitmap S.best over the n0 vertices of S.orig.
template <int SN>
__device__ void exact_rounds(Scratch &S, WarpSmem<SN> &sm, int n0, long long arcs, long long &lam, int &err,
                             int &ovf, u64 seed, u64 tag, int pr_level, int fifo) {
    const int lane = lane_id();
    int n = n0;
    int *rpA = S.rpA, *srcA = S.srcA, *rpB = S.rpB, *srcB = S.srcB;
    int2 *adjA = S.adjA, *adjB = S.adjB;
    int round = 0, guard = 0;
    while (!err && n >= 2 && lam > 0) {
        if (++guard > 4 * n0 + 16) { err = MC_EINTERNAL; break; }
        const bool chip = round_on_chip<SN>(n, lam, fifo);
        unsigned short *par16 = chip ? sm.u.s.par : nullptr;
        // on chip the PR unions run on 32-bit parents in r (idle until the
        // scan), then pass to the 16-bit parents the scan's joins extend
        int *par32 = chip ? sm.r : S.par;
        for (int v = lane; v < n; v += 32) par32[v] = v;
        __syncwarp();
        long long un = 0;
        // Padberg-Rinaldi PR1/PR2 and the degree-2 tie rule
        if (pr_level >= 1) un = pr_unions(par32, rpA, srcA, adjA, S.deg, n, arcs, lam, pr_level);
        if (chip) {
            for (int v = lane; v < n; v += 32) par16[v] = (unsigned short)par32[v];
            __syncwarp();
        }
        // one full capped CAPFOREST scan
        ScanArgs A;
        A.g.n = n; A.g.arcs = arcs; A.g.rp = rpA; A.g.src = srcA; A.g.adj = adjA; A.g.deg = S.deg;
        A.par = S.par; A.T = S.T; A.order = S.order; A.st = S.st;
        A.rec_alpha = S.rec_alpha; A.rec_len = S.rec_len; A.perm_a = 1; A.perm_b = 0; A.limit = 0;
        const u64 h = splitmix64(seed ^ splitmix64((tag << 20) ^ (u64)round));
        const int start = (int)(h % (u64)n);
        Counters cnt;
        warp_full_scan<SN>(A, sm, S, n, arcs, lam, start, fifo, par16, cnt);
        un += cnt.unions;
        un = warp_sum_ll(un);
        const long long lam2 = ld_volatile_i64(&S.st->lam);
        if (lam2 < lam) {
            const int len = S.rec_len[1];
            warp_side_bits(S.best, n0, [&](int v) {
                const int c = S.orig[v];
                return S.T[c] == 1 && S.order[c] < len;
            });
            lam = lam2;
            if (un == 0) { ++round; continue; }
        }
        if (un == 0) { err = MC_EINTERNAL; break; }
        // contraction
        const int nc = chip ? warp_relabel(par16, S.root, S.lab, S.cnt, n) : warp_relabel(S.par, S.root, S.lab, S.cnt, n);
        // the result goes to the B buffers, then A and B swap roles
        if (n <= SN)
            arcs = warp_contract_chip<SN>(srcA, adjA, arcs, S.lab, n, nc, lam, S.rpT, S.adjT, rpB, srcB, adjB,
                                          S.deg, sm, &ovf);
        else
            arcs = warp_contract(srcA, adjA, arcs, S.lab, nc, lam, S.rpT, S.adjT, rpB, srcB, adjB, S.deg, S.cnt,
                                 S.mark, &ovf);
        for (int v = lane; v < n0; v += 32) S.orig[v] = S.lab[S.orig[v]];
        __syncwarp();
        {
            int *t = rpA; rpA = rpB; rpB = t;
            t = srcA; srcA = srcB; srcB = t;
            int2 *ta = adjA; adjA = adjB; adjB = ta;
        }
        n = nc;
        if (n >= 2) {
            long long md;
            int arg;
            warp_min_deg(S.deg, n, &md, &arg);
            if (md < lam) {
                lam = md;
                warp_side_bits(S.best, n0, [&](int v) { return S.orig[v] == arg; });
            }
        }
        ++round;
    }
}

template <int SN>
__device__ void solve_one(const BatchIn &B, int gi, Scratch &S, WarpSmem<SN> &sm) {
    const int lane = lane_id();
    const long long v0 = B.voff[gi];
    const int n0 = (int)(B.voff[gi + 1] - v0);
    const int *rp_in = B.rp + v0 + gi;
    const long long a0 = B.aoff[gi];
    const int *col_in = B.col + a0, *w_in = B.w + a0;
    int err = 0;
    int ovf = 0;
    long long arcs = 0;

    // Input that is canonical as given (rows strictly increasing, no
    // self-loop, positive weights, neighbours in range) is copied into A in
    // one arc-parallel pass: each arc's row counted against 32 consecutive
    // row starts held one a lane (the offsets staged on chip when they fit),
    // the degrees by a segmented sum over the lanes of a row.  The same pass checks symmetry in row order: the
    // downward arcs (u -> v, v < u) that reach v, met in increasing u, must
    // match the entries of row v above v one by one (a cursor per row,
    // starting at the row's first entry above v), with equal weights, and
    // every cursor must end at its row's end; that pairs every arc with its
    // mirror.  The mirror loads of a chunk are independent of one another.
    // Each lane carries kCU arcs at once.  Other input takes the general
    // path below (drop, sort, merge, symmetry check).
    constexpr int kCU = 4;
    const int m_raw = __ldg(rp_in + n0);
    const bool rp_on_chip = n0 < SN;
    int *cur = rp_on_chip ? sm.u.s.rp : S.cnt;
    // staged, and checked: offsets from 0 to the arc count, never falling
    // (the host checked the ends; a falling offset makes the graph MC_EINVAL
    // before any of its arcs is read)
    bool rp_bad = false;
    int rprev = 0;  // the offset before this chunk
    for (int v0 = 0; v0 <= n0; v0 += 32) {
        const int v = v0 + lane;
        const int r = v <= n0 ? __ldg(rp_in + v) : INT_MAX;
        int pr = __shfl_up_sync(0xffffffffu, r, 1);
        if (lane == 0) pr = rprev;
        if (v <= n0) {
            if (r < pr || (v == 0 && r != 0)) rp_bad = true;
            S.rpA[v] = r;
            if (rp_on_chip) sm.r[v] = r;
            if (v > 0) cur[v - 1] = r;  // no entry above v-1 seen yet: the row's end
        }
        rprev = __shfl_sync(0xffffffffu, r, 31);
    }
    const bool rp_ok = !__any_sync(0xffffffffu, rp_bad);  // warp-uniform
    if (!rp_ok) err = MC_EINVAL;
    for (int v = lane; v < n0; v += 32) S.deg[v] = 0;
    __syncwarp();
    const int *rps = rp_on_chip ? sm.r : rp_in;
    int ucur = 0;  // a row starting at or before the window's first arc
    bool canon = m_raw >= 0 && rp_ok;
    bool sym_ok = true;
    int vn[kCU], cn[kCU];  // the next chunk's arcs, loaded one chunk ahead
#pragma unroll
    for (int j = 0; j < kCU; ++j) {
        const int i = 32 * j + lane;
        vn[j] = i < m_raw ? col_in[i] : -1;
        cn[j] = i < m_raw ? w_in[i] : 0;
    }
    for (int i0 = 0; i0 < m_raw && canon; i0 += 32 * kCU) {
        int u[kCU], v[kCU], c[kCU];
#pragma unroll
        for (int j = 0; j < kCU; ++j) {
            const int i = i0 + 32 * j + lane, ia = i + 32 * kCU;
            u[j] = i < m_raw ? 0 : -1;
            v[j] = vn[j];
            c[j] = cn[j];
            vn[j] = ia < m_raw ? col_in[ia] : -1;
            cn[j] = ia < m_raw ? w_in[ia] : 0;
        }
        const int prev0 = lane == 0 && i0 > 0 ? col_in[i0 - 1] : -1;
        // row of each arc: ucur plus the row starts in (ucur, i], counted
        // against 32 consecutive starts held one a lane (a 5-step search over
        // shuffles), 32 more while some arc lies past them
        {
            int base = ucur;
            unsigned pending = 0u;
#pragma unroll
            for (int j = 0; j < kCU; ++j)
                if (u[j] >= 0) pending |= 1u << j;
            while (__any_sync(0xffffffffu, pending != 0u)) {
                const int su = base + 1 + lane;
                const int st = su <= n0 ? rps[su] : INT_MAX;
                const int st31 = __shfl_sync(0xffffffffu, st, 31);
#pragma unroll
                for (int j = 0; j < kCU; ++j) {
                    const int i = i0 + 32 * j + lane;
                    int pos = 0;  // starts at or before i among the first 31
#pragma unroll
                    for (int b = 16; b > 0; b >>= 1)
                        if (__shfl_sync(0xffffffffu, st, pos + b - 1) <= i) pos += b;
                    if (pos == 31 && st31 <= i) pos = 32;
                    if (((pending >> j) & 1u) && pos < 32) {
                        u[j] = base + pos;
                        pending &= ~(1u << j);
                    }
                }
                base += 32;
            }
            const int lastu = __shfl_sync(0xffffffffu, u[kCU - 1], 31);
            if (lastu >= 0) ucur = lastu;
        }
        bool ok = true;
#pragma unroll
        for (int j = 0; j < kCU; ++j) {
            const int i = i0 + 32 * j + lane;
            int pv = __shfl_up_sync(0xffffffffu, v[j], 1);  // the previous arc's neighbour
            const int last = __shfl_sync(0xffffffffu, v[(j + kCU - 1) % kCU], 31);
            if (lane == 0) pv = j > 0 ? last : prev0;
            if (u[j] >= 0) {
                const bool row_first = i == rps[u[j]];
                ok = ok && v[j] >= 0 && v[j] < n0 && v[j] != u[j] && c[j] > 0 && (row_first || pv < v[j]);
                S.srcA[i] = u[j];
                S.adjA[i] = make_int2(v[j], c[j]);
                if (v[j] > u[j] && (row_first || pv < u[j])) cur[u[j]] = i;  // row u's first entry above u
            }
        }
        __syncwarp();
        // each downward arc takes the next entry above v in row v; lanes
        // meeting the same v are in row order, ranked by match_any
        int at[kCU], mv[kCU], mw[kCU];
#pragma unroll
        for (int j = 0; j < kCU; ++j) {
            const bool dn = u[j] >= 0 && v[j] >= 0 && v[j] < u[j];
            const unsigned peers = __match_any_sync(0xffffffffu, dn ? v[j] : -1 - lane);
            at[j] = -1;
            if (dn) at[j] = cur[v[j]] + __popc(peers & ((1u << lane) - 1u));
            __syncwarp();
            if (dn && (peers >> lane) == 1u) cur[v[j]] = at[j] + 1;
            __syncwarp();
            mv[j] = -1;
            mw[j] = 0;
            if (dn && at[j] < rps[v[j] + 1]) {
                mv[j] = col_in[at[j]];
                mw[j] = w_in[at[j]];
            }
        }
#pragma unroll
        for (int j = 0; j < kCU; ++j) {
            if (at[j] >= 0 && (mv[j] != u[j] || mw[j] != c[j])) sym_ok = false;
            // the lanes of one row add their weights toward its first lane
            long long cs = c[j];
            const int pu = __shfl_up_sync(0xffffffffu, u[j], 1);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long t = __shfl_down_sync(0xffffffffu, cs, o);
                const int tu = __shfl_down_sync(0xffffffffu, u[j], o);
                if (lane + o < 32 && tu == u[j]) cs += t;
            }
            if (u[j] >= 0 && (lane == 0 || pu != u[j]))
                atomicAdd(reinterpret_cast<unsigned long long *>(&S.deg[u[j]]), (unsigned long long)cs);
        }
        canon = __all_sync(0xffffffffu, ok);
    }
    if (canon) {
        arcs = m_raw;
        for (int x = lane; x < n0; x += 32)
            if (cur[x] != rps[x + 1]) sym_ok = false;  // an entry above x with no downward arc
        if (!__all_sync(0xffffffffu, sym_ok)) err = MC_EINVAL;
        __syncwarp();
    }

    // raw arcs -> (srcB, adjB), dropping self-loops and zero weights
    long long m = 0;
    for (int u = 0; u < n0 && !canon && rp_ok; ++u) {
        const int lo = rp_in[u], hi = rp_in[u + 1];
        for (int e0 = lo; e0 < hi; e0 += 32) {
            const int e = e0 + lane;
            bool keep = false;
            int v = 0, c = 0;
            if (e < hi) {
                v = col_in[e];
                c = w_in[e];
                if (v < 0 || v >= n0) err = MC_EINVAL;
                else if (c < 0) err = MC_EINVAL;
                else keep = v != u && c > 0;
            }
            const unsigned kb = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const long long pos = m + __popc(kb & ((1u << lane) - 1u));
                S.srcB[pos] = u;
                S.adjB[pos] = make_int2(v, c);
            }
            m += __popc(kb);
        }
    }
    err = __reduce_or_sync(0xffffffffu, err);
    if (!canon && !err) {
        // canonical CSR in A (identity labels)
        for (int v = lane; v < n0; v += 32) S.lab[v] = v;
        __syncwarp();
        arcs = warp_contract(S.srcB, S.adjB, m, S.lab, n0, kInt32Max, S.rpT, S.adjT, S.rpA, S.srcA, S.adjA, S.deg,
                             S.cnt, S.mark, &ovf);
        if (__reduce_or_sync(0xffffffffu, ovf)) err = MC_EOVERFLOW;
    }
    // an arc without its mirror (same weight after merging) is malformed
    // input: the raw-arc buffers (B) and the sort buffers (T) are free here
    if (!err && !canon &&
        !warp_symmetric(S.rpA, S.srcA, S.adjA, arcs, n0, S.rpT, S.srcB, S.adjB, S.rpB, S.eslot, S.adjT, S.cnt,
                        S.mark))
        err = MC_EINVAL;

    long long lam = 0;
    if (!err) {
        // no separate components pass: a disconnected graph's first scan
        // ends with its start's component, whose cut (alpha = 0) sets
        // lambda = 0 and the side; a vertex without arcs gives delta = 0
        int arg = 0;
        warp_min_deg(S.deg, n0, &lam, &arg);
        if (lam >= 0x7FFFFFFD) err = MC_EOVERFLOW;
        warp_side_bits(S.best, n0, [&](int v) { return v == arg; });
        for (int v = lane; v < n0; v += 32) S.orig[v] = v;
        __syncwarp();
        exact_rounds<SN>(S, sm, n0, arcs, lam, err, ovf, B.seed, (u64)gi, B.pr_level, B.fifo);
    }
    if (lane == 0) {
        B.lam_out[gi] = lam;
        B.err_out[gi] = err;
    }
    if (B.bits_out && !err) {
        u32 *dst = B.bits_out + B.bits_off[gi];
        const int nw = (n0 + 31) / 32;
        const bool flip = S.best[0] & 1u;
        for (int i = lane; i < nw; i += 32) {
            u32 v = flip ? ~S.best[i] : S.best[i];
            if (i == nw - 1 && (n0 & 31)) v &= (1u << (n0 & 31)) - 1u;
            dst[i] = v;
        }
    }
    __syncwarp();
}

template <int WPB, int SN>
__global__ void __launch_bounds__(WPB * 32) k_batch(BatchIn B) {
    __shared__ WarpSmem<SN> smem[WPB];
    const int wid = threadIdx.x >> 5;
    const int gw = blockIdx.x * WPB + wid;
    Scratch S0 = scratch_of(B.scratch + (size_t)gw * B.L.bytes, B.L);
    while (true) {
        int k = 0;
        if (lane_id() == 0) k = atomicAdd(B.next, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= B.G) break;
        solve_one<SN>(B, B.order[k], S0, smem[wid]);
    }
}

// ------------------------------------------------------------ tail solver --
constexpr int kTailSN = 2048;

struct TailIn {
    DevGraph g;
    long long lam;
    unsigned char *scratch;
    Layout L;
    u64 seed;
    int pr_level, fifo;
    Status *out;  // out->lam = the minimum found, out->err
    u32 *bits_out;  // if set: the side bitmap (n bits) is copied here
};

// one warp: copy the small graph into its scratch, then Alg. 2's rounds.
// SMEM_SCRATCH: the whole scratch (graph copies included) lives in dynamic
// shared memory, so every access of the rounds is on-chip.
template <int SN, bool SMEM_SCRATCH>
__global__ void __launch_bounds__(32) k_tail(TailIn T) {
    __shared__ WarpSmem<SN> sm;
    extern __shared__ __align__(256) unsigned char tail_smem[];
    Scratch S = scratch_of(SMEM_SCRATCH ? tail_smem : T.scratch, T.L);
    const int lane = lane_id();
    const int n = T.g.n;
    const long long arcs = T.g.arcs;
    for (int v = lane; v <= n; v += 32) S.rpA[v] = T.g.rp[v];
    for (int v = lane; v < n; v += 32) { S.deg[v] = T.g.deg[v]; S.orig[v] = v; }
    for (long long i = lane; i < arcs; i += 32) { S.srcA[i] = T.g.src[i]; S.adjA[i] = T.g.adj[i]; }
    __syncwarp();
    long long lam = T.lam;
    int err = 0, ovf = 0;
    exact_rounds<SN>(S, sm, n, arcs, lam, err, ovf, T.seed, 0x7A11ULL, T.pr_level, T.fifo);
    if (T.bits_out && lam < T.lam)
        for (int i = lane; i < (n + 31) / 32; i += 32) T.bits_out[i] = S.best[i];
    if (lane == 0) {
        T.out->lam = lam;
        T.out->err = err;
    }
}

// ------------------------------------------------------------ host side --
struct BatchCtx {
    unsigned char *scratch = nullptr;
    size_t scratch_bytes = 0;
    void *io = nullptr;
    size_t io_bytes = 0;
    cudaStream_t stream = nullptr;
    // the captured {reset the work counter, persistent launch} of the last
    // batch layout; replayed while the layout (and so every kernel
    // argument) is unchanged
    cudaGraphExec_t exec = nullptr;
    unsigned char key[sizeof(BatchIn) + 3 * sizeof(int)] = {};
    long long replays = 0;
};
std::mutex g_batch_mutex;
BatchCtx g_batch[64];

int grow(void **p, size_t *cur, size_t want, cudaStream_t s) {
    if (*cur >= want) return MC_OK;
    if (*p) {
        cudaStreamSynchronize(s);
        dev_free(*p, s);
        *p = nullptr;
        *cur = 0;
    }
    MC_TRY(dev_alloc(p, want, s));
    *cur = want;
    return MC_OK;
}

template <int WPB, int SN>
int launch_batch(const BatchIn &B, int warps, cudaStream_t s) {
    const int blocks = (warps + WPB - 1) / WPB;
    ++::mc::g_launches; k_batch<WPB, SN><<<blocks, WPB * 32, 0, s>>>(B);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

}  // namespace

// batch configurations the autotuner chooses from: warps per block x shared
// vertices per warp
// and whether the in-warp PR1/PR2 tests run (they never change a lambda;
// on small graphs the scans' own joins often make them cost more than they
// save, so the autotuner times both)
struct BatchShape {
    int wpb, sn;
    bool pr;
};
static const BatchShape kShapes[] = {{4, 1024, true},  {4, 2048, true},  {8, 512, true},  {8, 1024, true},
                                     {2, 2048, true},  {4, 1024, false}, {4, 2048, false}, {8, 512, false},
                                     {8, 1024, false}, {2, 2048, false}};
static int g_shape_choice = -1;  // -1: not tuned

static int run_batch(int shape, BatchIn B, int warps, cudaStream_t s) {
    const BatchShape sh = kShapes[shape];
    if (sh.wpb == 4 && sh.sn == 1024) return launch_batch<4, 1024>(B, warps, s);
    if (sh.wpb == 4 && sh.sn == 2048) return launch_batch<4, 2048>(B, warps, s);
    if (sh.wpb == 8 && sh.sn == 512) return launch_batch<8, 512>(B, warps, s);
    if (sh.wpb == 8 && sh.sn == 1024) return launch_batch<8, 1024>(B, warps, s);
    return launch_batch<2, 2048>(B, warps, s);
}

static int blocks_per_sm(int shape) {
    const BatchShape sh = kShapes[shape];
    int b = 0;
    cudaError_t e;
    if (sh.wpb == 4 && sh.sn == 1024) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<4, 1024>, 128, 0);
    else if (sh.wpb == 4 && sh.sn == 2048) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<4, 2048>, 128, 0);
    else if (sh.wpb == 8 && sh.sn == 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<8, 512>, 256, 0);
    else if (sh.wpb == 8 && sh.sn == 1024) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<8, 1024>, 256, 0);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch<2, 2048>, 64, 0);
    if (e != cudaSuccess) { (void)cudaGetLastError(); b = 1; }
    return b < 1 ? 1 : b;
}

int batch_solve(int G, const long long *vtx_off, const long long *arc_off, const int *row_ptr,
                const int *col, const int *w, const mc_options &o, long long *lambdas, u32 *bitmaps,
                const long long *bitmap_word_off, int shape, double *ms_out) {
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MC_EINVAL;
    std::lock_guard<std::mutex> lock(g_batch_mutex);
    BatchCtx &ctx = g_batch[dev];
    if (!ctx.stream) MC_CUDA(cudaStreamCreateWithFlags(&ctx.stream, cudaStreamNonBlocking));
    cudaStream_t s = o.cuda_stream ? static_cast<cudaStream_t>(o.cuda_stream) : ctx.stream;

    // host-side validation of the offsets
    int nmax = 0;
    long long amax = 0;
    for (int k = 0; k < G; ++k) {
        const long long n = vtx_off[k + 1] - vtx_off[k];
        const long long a = arc_off[k + 1] - arc_off[k];
        if (n < 2 || n > (1 << 24) || a < 0) return MC_EINVAL;
        const int *rp = row_ptr + vtx_off[k] + k;
        // the ends here; a falling offset inside is found by the kernel
        if (rp[0] != 0 || (long long)rp[n] != a) return MC_EINVAL;
        nmax = std::max(nmax, (int)n);
        amax = std::max(amax, a);
    }
    if (G == 0) return MC_OK;
    std::vector<int> order((size_t)G);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return arc_off[x + 1] - arc_off[x] > arc_off[y + 1] - arc_off[y];
    });

    if (shape < 0) shape = g_shape_choice >= 0 ? g_shape_choice : 0;
    const Layout L = make_layout(nmax, amax);
    const int wpb = kShapes[shape].wpb;
    const int warps_res = blocks_per_sm(shape) * wpb * num_sms();
    int warps = std::min(warps_res, G);
    warps = (warps + wpb - 1) / wpb * wpb;  // whole blocks: every warp owns a scratch slice

    // device copies of the inputs and outputs in one buffer
    const long long V = vtx_off[G], A = arc_off[G];
    const long long bw = bitmaps ? bitmap_word_off[G] : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t r = off; off += al(bytes); return r; };
    const size_t o_voff = take(8 * (G + 1)), o_aoff = take(8 * (G + 1)), o_rp = take(4 * (V + G)),
                 o_col = take(4 * (A > 0 ? A : 1)), o_w = take(4 * (A > 0 ? A : 1)),
                 o_ord = take(4 * G), o_lam = take(8 * G), o_err = take(4 * G),
                 o_bits = take(4 * (bw > 0 ? bw : 1)), o_boff = take(8 * (G + 1)), o_next = take(4);
    MC_TRY(grow(&ctx.io, &ctx.io_bytes, off, s));
    MC_TRY(grow(reinterpret_cast<void **>(&ctx.scratch), &ctx.scratch_bytes, L.bytes * (size_t)warps, s));
    unsigned char *io = static_cast<unsigned char *>(ctx.io);
    MC_CUDA(cudaMemcpyAsync(io + o_voff, vtx_off, 8 * (G + 1), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(io + o_aoff, arc_off, 8 * (G + 1), cudaMemcpyHostToDevice, s));
    MC_CUDA(cudaMemcpyAsync(io + o_rp, row_ptr, 4 * (V + G), cudaMemcpyHostToDevice, s));
    if (A > 0) {
        MC_CUDA(cudaMemcpyAsync(io + o_col, col, 4 * A, cudaMemcpyHostToDevice, s));
        MC_CUDA(cudaMemcpyAsync(io + o_w, w, 4 * A, cudaMemcpyHostToDevice, s));
    }
    MC_CUDA(cudaMemcpyAsync(io + o_ord, order.data(), 4 * (size_t)G, cudaMemcpyHostToDevice, s));
    if (bitmaps) MC_CUDA(cudaMemcpyAsync(io + o_boff, bitmap_word_off, 8 * (G + 1), cudaMemcpyHostToDevice, s));


    BatchIn B;
    B.G = G;
    B.voff = (const long long *)(io + o_voff);
    B.aoff = (const long long *)(io + o_aoff);
    B.rp = (const int *)(io + o_rp);
    B.col = (const int *)(io + o_col);
    B.w = (const int *)(io + o_w);
    B.order = (const int *)(io + o_ord);
    B.lam_out = (long long *)(io + o_lam);
    B.err_out = (int *)(io + o_err);
    B.bits_out = bitmaps ? (u32 *)(io + o_bits) : nullptr;
    B.bits_off = bitmaps ? (const long long *)(io + o_boff) : nullptr;
    B.next = (int *)(io + o_next);
    B.scratch = ctx.scratch;
    B.L = L;
    B.seed = o.seed;
    B.pr_level = kShapes[shape].pr ? o.pr_level : 0;
    B.fifo = o.pq_order == MC_PQ_FIFO;

    cudaEvent_t ea, eb;
    cudaEventCreate(&ea);
    cudaEventCreate(&eb);
    // one persistent launch under a captured CUDA graph (re-captured when
    // the batch layout changes)
    int rc = MC_OK;
    {
        unsigned char key[sizeof(ctx.key)];
        memcpy(key, &B, sizeof(BatchIn));
        const int extra[3] = {shape, warps, (int)(o.cuda_stream != nullptr)};
        memcpy(key + sizeof(BatchIn), extra, sizeof(extra));
        if (!ctx.exec || memcmp(key, ctx.key, sizeof(key)) != 0) {
            if (ctx.exec) { cudaGraphExecDestroy(ctx.exec); ctx.exec = nullptr; }
            cudaGraph_t graph = nullptr;
            MC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            cudaError_t ce = cudaMemsetAsync(io + o_next, 0, 4, s);
            if (ce == cudaSuccess) rc = run_batch(shape, B, warps, s);
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            if (ce != cudaSuccess || ee != cudaSuccess || rc != MC_OK) {
                if (graph) cudaGraphDestroy(graph);
                if (rc != MC_OK) return rc;
                set_cuda_error(ce != cudaSuccess ? ce : ee, "batch graph capture");
                return MC_ECUDA;
            }
            cudaError_t ie = cudaGraphInstantiate(&ctx.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                ctx.exec = nullptr;
                set_cuda_error(ie, "cudaGraphInstantiate(batch)");
                return MC_ECUDA;
            }
            memcpy(ctx.key, key, sizeof(key));
        } else {
            ++ctx.replays;
        }
    }
    cudaEventRecord(ea, s);
    MC_CUDA(cudaGraphLaunch(ctx.exec, s));
    cudaEventRecord(eb, s);
    if (rc != MC_OK) {
        cudaEventDestroy(ea);
        cudaEventDestroy(eb);
        return rc;
    }
    std::vector<int> errs((size_t)G);
    MC_CUDA(cudaMemcpyAsync(lambdas, io + o_lam, 8 * (size_t)G, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaMemcpyAsync(errs.data(), io + o_err, 4 * (size_t)G, cudaMemcpyDeviceToHost, s));
    if (bitmaps) MC_CUDA(cudaMemcpyAsync(bitmaps, io + o_bits, 4 * bw, cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    cudaEventElapsedTime(&ms, ea, eb);
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (ms_out) *ms_out = ms;
    for (int k = 0; k < G; ++k)
        if (errs[k]) return errs[k];
    return MC_OK;
}

// graphs up to kTailSmemN vertices and kTailSmemArcs arcs run with the whole
// scratch in shared memory
constexpr int kTailSmemN = 256;
constexpr int kTailSmemArcs = 4096;
constexpr int kTailSmemSN = 256;

int tail_solve(const DevGraph &g, Work &w, int limit, long long *lam, u64 seed, int pr_level, int fifo,
               int n0, cudaStream_t s) {
    if (limit > 4096) limit = 4096;
    if (g.n > limit || g.arcs > 64LL * limit || g.n < 2) return MC_EINVAL;
    const bool on_chip = g.n <= kTailSmemN && g.arcs <= kTailSmemArcs;
    const Layout L = on_chip ? make_layout(kTailSmemN, kTailSmemArcs) : make_layout(limit, 64LL * limit);
    // the side bitmap is read back from global memory in both cases
    const size_t need = on_chip ? al(4 * ((size_t)kTailSmemN / 32 + 2)) : L.bytes;
    if (w.tail_bytes < need || !w.tail) {
        dev_free(w.tail, s);
        w.tail = nullptr;
        w.tail_bytes = 0;
        MC_TRY(dev_alloc(reinterpret_cast<void **>(&w.tail), need, s));
        w.tail_bytes = need;
    }
    TailIn T;
    T.g = g;
    T.lam = *lam;
    T.scratch = w.tail;
    T.L = L;
    T.seed = seed;
    T.pr_level = pr_level;
    T.fifo = fifo;
    T.out = w.st;
    T.bits_out = on_chip ? reinterpret_cast<u32 *>(w.tail) : nullptr;
    if (on_chip) {
        static bool attr = false;
        if (!attr) {
            MC_CUDA(cudaFuncSetAttribute(k_tail<kTailSmemSN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.bytes));
            attr = true;
        }
        ++::mc::g_launches; k_tail<kTailSmemSN, true><<<1, 32, L.bytes, s>>>(T);
    } else {
        ++::mc::g_launches; k_tail<kTailSN, false><<<1, 32, 0, s>>>(T);
    }
    MC_CUDA(cudaGetLastError());
    MC_TRY(status_read(w, s));
    if (w.h_st->err) {
        set_error_detail("tail solver failed");
        return w.h_st->err;
    }
    if (w.h_st->lam < *lam) {
        const u32 *bits = on_chip ? reinterpret_cast<const u32 *>(w.tail)
                                  : reinterpret_cast<const u32 *>(w.tail + L.best);
        MC_TRY(side_from_bits(w, n0, bits, s));
        *lam = w.h_st->lam;
    }
    return MC_OK;
}

int batch_shapes() { return (int)(sizeof(kShapes) / sizeof(kShapes[0])); }
void batch_set_shape(int shape) { g_shape_choice = shape; }
int batch_get_shape() { return g_shape_choice; }

}  // namespace mc
