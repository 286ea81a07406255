// mc_graph.cu -- graph ingest, contraction and bookkeeping kernels.
//
// Contraction (Sec. 2.1; Sec. 3.2 "Parallel Graph Contraction"): the paper
// builds G_C with a concurrent hash table keyed by the block ids of each
// edge.  Here the same G_C comes from
//   flatten the union-find -> number the blocks by a scan (block id order =
//   smallest member) -> emit one (block(u), block(v), c) arc per arc whose
//   ends fall in different blocks -> LSD radix sort on the packed key ->
//   segmented sum of parallel arcs -> CSR offsets, degrees and the minimum
//   degree (the lambda-hat update of Sec. 3.2).
// Merged weights are clamped to the current lambda-hat before the int32
// store: an edge of weight >= lambda-hat already certifies every cut through
// it is >= lambda-hat, so the clamp changes no cut below lambda-hat.
#include <cstdio>

#include <functional>

#include "mc_internal.cuh"
#include "mc_sort.cuh"

namespace mc {

constexpr int kThreads = 256;

static int grid_for(i64 n, int threads = kThreads) {
    i64 b = (n + threads - 1) / threads;
    i64 cap = (i64)num_sms() * 16;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// -------------------------------------------------------------- alloc ----
int graph_alloc(DevGraph &g, i64 n, i64 arcs, cudaStream_t s) {
    MC_TRY(dev_alloc_n(&g.rp, (size_t)n + 1, s));
    MC_TRY(dev_alloc_n(&g.src, (size_t)arcs, s));
    MC_TRY(dev_alloc_n(&g.adj, (size_t)arcs, s));
    MC_TRY(dev_alloc_n(&g.deg, (size_t)n, s));
    return MC_OK;
}

void graph_free(DevGraph &g, cudaStream_t s) {
    dev_free(g.rp, s); dev_free(g.src, s); dev_free(g.adj, s); dev_free(g.deg, s);
    g = DevGraph();
}

int work_alloc(Work &w, i64 n0, i64 arcs0, cudaStream_t s) {
    w.cap_n = n0;
    w.cap_arcs = arcs0;
    i64 a = arcs0 > n0 ? arcs0 : n0;
    MC_TRY(dev_alloc_n(&w.par, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.root, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.lab, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.T, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.order, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.cnt, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.orig, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.red, (size_t)kRedWords, s));
    MC_CUDA(cudaMemsetAsync(w.red, 0, sizeof(i64) * (size_t)kRedWords, s));
    MC_TRY(dev_alloc_n(&w.scan_tmp, scan_tmp_words(a * 256), s));
    MC_TRY(scan_tmp_clear(w.scan_tmp, scan_tmp_words(a * 256), s));
    MC_TRY(dev_alloc_n(&w.keysA, (size_t)a, s));
    MC_TRY(dev_alloc_n(&w.keysB, (size_t)a, s));
    MC_TRY(dev_alloc_n(&w.valsA, (size_t)a, s));
    MC_TRY(dev_alloc_n(&w.valsB, (size_t)a, s));
    MC_TRY(dev_alloc_n(&w.radix_tmp, radix_tmp_words(a), s));
    MC_TRY(dev_alloc_n(&w.rec_alpha, (size_t)n0 + 1, s));
    MC_TRY(dev_alloc_n(&w.rec_len, (size_t)n0 + 1, s));
    MC_TRY(dev_alloc_n(&w.fb_r, (size_t)n0, s));
    MC_TRY(dev_alloc_n(&w.fb_pool, 2 * ((size_t)a + 64), s));
    MC_TRY(dev_alloc_n(&w.best_side, (size_t)(n0 + 31) / 32, s));
    MC_TRY(dev_alloc_n(&w.st, 1, s));
    MC_CUDA(cudaMallocHost(reinterpret_cast<void **>(&w.h_st), sizeof(Status)));
    return MC_OK;
}

void work_free(Work &w, cudaStream_t s) {
    void *ps[] = {w.par, w.root, w.lab, w.T, w.order, w.cnt, w.orig, w.red, w.scan_tmp, w.keysA, w.keysB,
                  w.valsA, w.valsB, w.radix_tmp, w.rec_alpha, w.rec_len, w.fb_r, w.fb_pool,
                  w.best_side, w.st, w.tail, w.blk};
    for (void *p : ps) dev_free(p, s);
    if (w.h_st) cudaFreeHost(w.h_st);
    w = Work();
}

// ------------------------------------------------------------ helpers ----
__global__ void k_iota(int *a, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

int union_find_init(int *par, int n, cudaStream_t s) {
    ++::mc::g_launches; k_iota<<<grid_for(n), kThreads, 0, s>>>(par, n);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// flatten: root[v] = root of v in par; cnt[v] = (v is a root).  par is not
// written here, so the walks read it through the read-only cache (measured
// against path-halving finds on RHG 2^20: solve 1.79 -> 1.72 ms); the roots
// go to their own array.
__global__ void k_flatten(const int *__restrict__ par, int *__restrict__ root, int *__restrict__ cnt, int n, Status *st) {
    if (st && blockIdx.x == 0 && threadIdx.x == 0) st->count2 = 0;  // the emit counter
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int r = v, p = __ldg(par + v);
        while (p != r) { r = p; p = __ldg(par + r); }
        cnt[v] = (r == v);
        root[v] = r;
    }
}

// lab[v] = lab[root(v)]; roots already hold their new id from the scan
__global__ void k_relabel(const int *__restrict__ root, int *lab, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int r = root[v];
        if (r != v) lab[v] = lab[r];
    }
}

// ------------------------------------------------------------- emitting ---
// Block-chunked compaction: each block takes chunks of kEmitItems x 256 arcs,
// keeps its survivors in registers, ranks them with one block scan and
// reserves their output range with a single atomic per chunk (a per-warp
// atomic on one global counter serialises millions of times).
constexpr int kEmitItems = 4;
constexpr int kEmitChunk = kEmitItems * kThreads;

__device__ __forceinline__ int block_excl_scan_256(int v, int *total) {
    __shared__ int ws[kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int x = lane < kThreads / 32 ? ws[lane] : 0;
        int xs = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, xs, o);
            if (lane >= o) xs += t;
        }
        if (lane < kThreads / 32) ws[lane] = xs - x;
        if (lane == kThreads / 32 - 1) *total = xs;
    }
    __syncthreads();
    const int r = ws[wid] + inc - v;
    __syncthreads();
    return r;
}

// one (block(u), block(v), c) arc per arc with different blocks.  Within a
// warp's 32 consecutive arcs, a run of equal (block(u), block(v)) keys is
// emitted once by its first lane with the run's weight added up, saturated at
// min(clamp, INT32_MAX): the later segmented sum of saturated parts,
// saturated again, equals the saturated total.  wb > 0: the weight (at most
// min(clamp, INT32_MAX) < 2^wb) rides in the low wb bits of the key word,
// (key << wb) | weight, and vals is not written.
__global__ void __launch_bounds__(kThreads)
k_emit(const int *__restrict__ src, const int2 *__restrict__ adj, i64 arcs, const int *__restrict__ lab,
       u64 nc, const int *d_nc, i64 clamp, int wb, u64 *__restrict__ keys, int *__restrict__ vals,
       u64 *counter, int *err) {
    __shared__ int total;
    __shared__ u64 base_s;
    if (d_nc) nc = (u64)*d_nc;
    const long long cap = clamp < (i64)kInt32Max ? clamp : (i64)kInt32Max;
    const int lane = threadIdx.x & 31;
    for (i64 c0 = (i64)blockIdx.x * kEmitChunk; c0 < arcs; c0 += (i64)gridDim.x * kEmitChunk) {
        u64 key[kEmitItems];
        int val[kEmitItems];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kEmitItems; ++k) {
            const i64 i = c0 + (i64)k * kThreads + threadIdx.x;
            u64 kk = ~0ULL;
            long long c = 0;
            if (i < arcs) {
                const int2 e = adj[i];
                const int a = lab[src[i]], b = lab[e.x];
                if (a != b) {
                    kk = (u64)a * nc + (u64)b;
                    c = e.y;
                }
            }
            // runs of equal keys among the warp's lanes: saturating sums
            // (both terms <= cap < 2^31, so the u32 add cannot wrap) toward
            // the run's first lane; a lane takes lane + o's partial sum when
            // no run starts in (lane, lane + o]
            key[k] = ~0ULL;
            // after a round that contracted much, most warps hold no
            // crossing arc: nothing to merge
            if (!__any_sync(0xffffffffu, kk != ~0ULL)) continue;
            const u64 kp = __shfl_up_sync(0xffffffffu, kk, 1);
            // no lane continues a run of its left neighbour (the common
            // case): every crossing arc is emitted as it is
            if (!__any_sync(0xffffffffu, kk != ~0ULL && lane > 0 && kp == kk)) {
                if (kk != ~0ULL) {
                    if (c > cap && clamp > (i64)kInt32Max) atomicOr(err, kErrOverflow);
                    key[k] = kk;
                    val[k] = (int)(c > cap ? cap : c);
                    ++cnt;
                }
                continue;
            }
            const bool head = lane == 0 || kp != kk;
            const unsigned hm = __ballot_sync(0xffffffffu, head);
            const unsigned after = lane == 31 ? 0u : hm >> (lane + 1);
            bool wide = c > cap;
            unsigned sv = (unsigned)(c > cap ? cap : c);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned t = __shfl_down_sync(0xffffffffu, sv, o);
                if (lane + o < 32 && (after & ((1u << o) - 1u)) == 0) {
                    const unsigned x = sv + t;
                    wide |= x > (unsigned)cap;
                    sv = x > (unsigned)cap ? (unsigned)cap : x;
                }
            }
            if (head && kk != ~0ULL) {
                if (wide && clamp > (i64)kInt32Max) atomicOr(err, kErrOverflow);
                key[k] = kk;
                val[k] = (int)sv;
                ++cnt;
            }
        }
        const int off = block_excl_scan_256(cnt, &total);
        if (threadIdx.x == 0) base_s = total ? atomicAdd(counter, (u64)total) : 0;
        __syncthreads();
        u64 pos = base_s + off;
#pragma unroll
        for (int k = 0; k < kEmitItems; ++k)
            if (key[k] != ~0ULL) {
                if (wb) {
                    keys[pos] = (key[k] << wb) | (u64)(unsigned)val[k];
                } else {
                    keys[pos] = key[k];
                    vals[pos] = val[k];
                }
                ++pos;
            }
        __syncthreads();
    }
}

// raw input arcs: validate and emit (u, v, c) for u != v, c > 0 (w == nullptr:
// every arc has weight 1)
__global__ void __launch_bounds__(kThreads)
k_emit_raw(const int *__restrict__ rp, const int *__restrict__ col, const int *__restrict__ w, int n,
           i64 arcs, u64 *__restrict__ keys, int *__restrict__ vals, u64 *counter, int *err) {
    __shared__ int total;
    __shared__ u64 base_s;
    for (i64 c0 = (i64)blockIdx.x * kEmitChunk; c0 < arcs; c0 += (i64)gridDim.x * kEmitChunk) {
        u64 key[kEmitItems];
        int val[kEmitItems];
        int cnt = 0;
        // source row: largest u with rp[u] <= i, by binary search
        int u = 0;
        {
            int lo = 0, hi = n - 1;
            const i64 first = c0 + threadIdx.x;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((i64)rp[mid] <= first) lo = mid; else hi = mid - 1;
            }
            u = lo;
        }
#pragma unroll
        for (int k = 0; k < kEmitItems; ++k) {
            const i64 i = c0 + (i64)k * kThreads + threadIdx.x;
            key[k] = ~0ULL;
            if (i < arcs) {
                if (u + 1 < n && (i64)rp[u + 1] <= i) {  // rows are non-decreasing: search past u
                    int lo = u + 1, hi = n - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((i64)rp[mid] <= i) lo = mid; else hi = mid - 1;
                    }
                    u = lo;
                }
                const int v = col[i], c = w ? w[i] : 1;
                if (v < 0 || v >= n) atomicOr(err, kErrRange);
                else if (c < 0) atomicOr(err, kErrNegW);
                else if (u != v && c > 0) {
                    key[k] = (u64)u * (u64)n + (u64)v;
                    val[k] = c;
                    ++cnt;
                }
            }
        }
        const int off = block_excl_scan_256(cnt, &total);
        if (threadIdx.x == 0) base_s = total ? atomicAdd(counter, (u64)total) : 0;
        __syncthreads();
        u64 pos = base_s + off;
#pragma unroll
        for (int k = 0; k < kEmitItems; ++k)
            if (key[k] != ~0ULL) { keys[pos] = key[k]; vals[pos] = val[k]; ++pos; }
        __syncthreads();
    }
}

__global__ void k_check_rp(const int *__restrict__ rp, int n, int *err) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (rp[v + 1] < rp[v]) atomicOr(err, kErrRange);
        if (v == 0 && rp[0] != 0) atomicOr(err, kErrRange);
    }
}

// ------------------------------------------------------ segmented sum ----
// (keys packed with a wb-bit weight compare above it)
__global__ void k_heads(const u64 *__restrict__ keys, i64 m, int wb, int *__restrict__ flag) {
    for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (i64)gridDim.x * blockDim.x)
        flag[i] = (i == 0) || ((keys[i] >> wb) != (keys[i - 1] >> wb));
}

// sum the weights of each run of equal keys into acc[j] (int64), write the
// run's (src, col); `ex` is the exclusive scan of the head flags.  wb > 0:
// the weights are the low wb bits of the key words (vals unused).
__global__ void k_seg_sum(const u64 *__restrict__ keys, const int *__restrict__ vals, int wb,
                          const int *__restrict__ ex, i64 m, u64 nc, u64 *__restrict__ acc,
                          int *__restrict__ osrc, int2 *__restrict__ oadj) {
    const int lane = threadIdx.x & 31;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    for (i64 i0 = (i64)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < m; i0 += stride) {
        i64 i = i0 + lane;
        bool ok = i < m;
        const u64 word = ok ? keys[i] : ~0ULL;
        const u64 key = word >> wb;
        bool head = ok && (i == 0 || (keys[i - 1] >> wb) != key);
        long long j = ok ? (long long)ex[i] + (head ? 1 : 0) - 1 : -1 - lane;
        long long s = !ok ? 0 : wb ? (long long)(word & ((1ULL << wb) - 1ULL)) : (long long)vals[i];
        // segmented reduction toward the first lane of each run in this warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_down_sync(0xffffffffu, s, o);
            long long jo = __shfl_down_sync(0xffffffffu, j, o);
            if (lane + o < 32 && jo == j) s += t;
        }
        long long jp = __shfl_up_sync(0xffffffffu, j, 1);
        bool first = ok && (lane == 0 || jp != j);
        if (first) atomicAdd(&acc[j], (u64)s);
        if (head) {
            osrc[j] = (int)(key / nc);
            oadj[j].x = (int)(key % nc);
        }
    }
}

// clamp the summed weights, store them, and accumulate degrees
__global__ void k_finalize(const u64 *__restrict__ acc, const int *d_m, i64 clamp, const int *__restrict__ osrc,
                           int2 *__restrict__ oadj, unsigned long long *deg, int *err) {
    const int lane = threadIdx.x & 31;
    const i64 m = *d_m;
    const i64 stride = (i64)gridDim.x * blockDim.x;
    for (i64 i0 = (i64)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < m; i0 += stride) {
        i64 i = i0 + lane;
        bool ok = i < m;
        long long s = ok ? (long long)acc[i] : 0;
        if (s > clamp) s = clamp;
        if (ok && s > kInt32Max) { atomicOr(err, kErrOverflow); s = kInt32Max; }
        int a = ok ? osrc[i] : -1 - lane;
        if (ok) oadj[i].y = (int)s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_down_sync(0xffffffffu, s, o);
            int ao = __shfl_down_sync(0xffffffffu, a, o);
            if (lane + o < 32 && ao == a) s += t;
        }
        int ap = __shfl_up_sync(0xffffffffu, a, 1);
        if (ok && (lane == 0 || ap != a)) atomicAdd(&deg[a], (unsigned long long)s);
    }
}

// CSR offsets from the sorted sources
__global__ void k_rowptr(const int *__restrict__ osrc, const int *d_m, int nc, int *__restrict__ rp) {
    const i64 m = d_m ? *d_m : 0;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j <= m; j += (i64)gridDim.x * blockDim.x) {
        int prev = j == 0 ? -1 : osrc[j - 1];
        int cur = j == m ? nc : osrc[j];
        for (int x = prev + 1; x <= cur && x <= nc; ++x) rp[x] = (int)j;
        if (j == m && m == 0) rp[nc] = 0;
    }
}

// ------------------------------------------------------------ min degree --
// minimum weighted degree and the smallest vertex with it, in one launch:
// each block reduces its vertices to (degree, vertex), and the last block to
// finish reduces the blocks' pairs (its counter comes back to 0)
__device__ __forceinline__ void md_better(long long &d, int &v, long long d2, int v2) {
    if (d2 < d || (d2 == d && v2 < v)) { d = d2; v = v2; }
}

// thread 0 ends with the block's best pair
__device__ void md_block_reduce(long long &d, int &v) {
    __shared__ long long sd[kThreads / 32];
    __shared__ int sv[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        md_better(d, v, __shfl_xor_sync(0xffffffffu, d, o), __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) { sd[threadIdx.x >> 5] = d; sv[threadIdx.x >> 5] = v; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 1; k < kThreads / 32; ++k) md_better(d, v, sd[k], sv[k]);
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads)
k_min_deg(const i64 *__restrict__ deg, int n, Status *st, long long *part, unsigned *done) {
    __shared__ bool last;
    long long d = LLONG_MAX;
    int v = INT_MAX;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        md_better(d, v, deg[u], u);
    md_block_reduce(d, v);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = d;
        part[2 * blockIdx.x + 1] = v;
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    d = LLONG_MAX;
    v = INT_MAX;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        md_better(d, v, *(volatile long long *)&part[2 * b], (int)*(volatile long long *)&part[2 * b + 1]);
    md_block_reduce(d, v);
    if (threadIdx.x == 0) {
        st->mindeg = d;
        st->argmin = v;
        *done = 0;
    }
}

int min_degree(const DevGraph &g, Work &w, cudaStream_t s) {
    int blocks = grid_for(g.n);
    if (blocks > kMinDegBlocks) blocks = kMinDegBlocks;
    ++::mc::g_launches;
    k_min_deg<<<blocks, kThreads, 0, s>>>(g.deg, g.n, w.st, w.red, reinterpret_cast<unsigned *>(w.red + kRedMinDone));
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

__global__ void k_zero_count(Status *st) {
    st->count = 0;
    st->count2 = 0;
}

// largest arc weight (st->count) and number of rows with exactly two arcs
// (st->count2): when max weight < lambda-hat, 2 * max weight <= delta and no
// row has two arcs, PR1, PR2 and the degree-2 rule cannot unite anything
__global__ void k_graph_stats(const DevGraph g, Status *st) {
    int wmax = 0;
    long long two = 0;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < g.arcs; j += (i64)gridDim.x * blockDim.x)
        wmax = max(wmax, g.adj[j].y);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < g.n; v += gridDim.x * blockDim.x)
        two += g.rp[v + 1] - g.rp[v] == 2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        two += __shfl_xor_sync(0xffffffffu, two, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (wmax) atomicMax(reinterpret_cast<unsigned long long *>(&st->count), (unsigned long long)wmax);
        if (two) atomicAdd(reinterpret_cast<unsigned long long *>(&st->count2), (unsigned long long)two);
    }
}

int graph_stats(const DevGraph &g, Work &w, cudaStream_t s) {
    ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(w.st);
    ++::mc::g_launches; k_graph_stats<<<grid_for(g.arcs > g.n ? g.arcs : g.n), kThreads, 0, s>>>(g, w.st);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

static int bits_for(u64 x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

// sorted (keys, vals) of m arcs over nc vertices -> out graph (+ degrees).
// The merged arc count stays on the device until the one status read at the
// end; `post` (may be empty) launches more work before that read.
// wb > 0: the pairs are packed words (key << wb) | weight, sorted keys only.
static int build_from_pairs(i64 m, int nc, i64 clamp, int wb, DevGraph &out, Work &w, cudaStream_t s,
                            const std::function<int()> &post) {
    bool in_b = false;
    if (wb)
        MC_TRY(radix_sort_keys(w.keysA, w.keysB, m, wb, bits_for((u64)nc * (u64)nc - 1), w.radix_tmp, w.scan_tmp,
                               &w.st->err, &in_b, s));
    else
        MC_TRY(radix_sort_pairs(w.keysA, w.valsA, w.keysB, w.valsB, m, bits_for((u64)nc * (u64)nc - 1),
                                w.radix_tmp, w.scan_tmp, &w.st->err, &in_b, s));
    u64 *keys = in_b ? w.keysB : w.keysA;
    int *vals = in_b ? w.valsB : w.valsA;
    int *flags = in_b ? w.valsA : w.valsB;      // free int32 buffer
    u64 *acc = in_b ? w.keysA : w.keysB;        // free 64-bit buffer
    int *d_total = reinterpret_cast<int *>(&w.st->count2);
    MC_CUDA(cudaMemsetAsync(&w.st->count2, 0, sizeof(w.st->count2), s));
    MC_CUDA(cudaMemsetAsync(out.deg, 0, sizeof(i64) * (size_t)nc, s));
    if (m > 0) {
        ++::mc::g_launches; k_heads<<<grid_for(m), kThreads, 0, s>>>(keys, m, wb, flags);
        MC_TRY(exclusive_scan_i32(flags, flags, m, d_total, w.scan_tmp, &w.st->err, s));
        MC_CUDA(cudaMemsetAsync(acc, 0, sizeof(u64) * (size_t)m, s));
        ++::mc::g_launches; k_seg_sum<<<grid_for(m), kThreads, 0, s>>>(keys, vals, wb, flags, m, (u64)nc, acc, out.src,
                                                   out.adj);
        ++::mc::g_launches; k_finalize<<<grid_for(m), kThreads, 0, s>>>(acc, d_total, clamp, out.src, out.adj,
                                                    reinterpret_cast<unsigned long long *>(out.deg),
                                                    &w.st->err);
    }
    ++::mc::g_launches; k_rowptr<<<grid_for(m + 1), kThreads, 0, s>>>(out.src, m > 0 ? d_total : nullptr, nc, out.rp);
    MC_CUDA(cudaGetLastError());
    out.n = nc;
    if (post) MC_TRY(post());
    MC_TRY(status_read(w, s));
    out.arcs = m > 0 ? (i64)(int)w.h_st->count2 : 0;
    return MC_OK;
}

int contract_graph(const DevGraph &in, DevGraph &out, Work &w, i64 clamp, bool flatten, int nc,
                   cudaStream_t s, const std::function<int()> &post) {
    const int n = in.n;
    // count2 (the emitted arcs) starts at 0: zeroed by the flatten, else here
    if (!flatten) { ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(w.st); }
    const int *d_nc = nullptr;
    if (flatten) {
        ++::mc::g_launches; k_flatten<<<grid_for(n), kThreads, 0, s>>>(w.par, w.root, w.cnt, n, w.st);
        d_nc = reinterpret_cast<int *>(&w.st->count);
        MC_TRY(exclusive_scan_i32(w.cnt, w.lab, n, reinterpret_cast<int *>(&w.st->count), w.scan_tmp, &w.st->err, s));
        ++::mc::g_launches; k_relabel<<<grid_for(n), kThreads, 0, s>>>(w.root, w.lab, n);
    }
    // pack the emitted weight under the block pair when both fit one word
    // (blocks <= n, weights <= min(clamp, INT32_MAX)): the sort then moves
    // 8 bytes an arc instead of 12
    const i64 cap = clamp < (i64)kInt32Max ? clamp : (i64)kInt32Max;
    const int wb = bits_for((u64)(cap > 1 ? cap : 1));
    const int pack = (n >= 2 && bits_for((u64)n * (u64)n - 1) + wb <= 64) ? wb : 0;
    // block count (device) and emitted arcs in one status read
    ++::mc::g_launches; k_emit<<<grid_for((in.arcs + kEmitItems - 1) / kEmitItems), kThreads, 0, s>>>(
        in.src, in.adj, in.arcs, w.lab, (u64)nc, d_nc, clamp, pack, w.keysA, w.valsA,
        reinterpret_cast<u64 *>(&w.st->count2), &w.st->err);
    MC_CUDA(cudaGetLastError());
    MC_TRY(status_read(w, s));
    if (flatten) nc = (int)w.h_st->count;
    const i64 m = w.h_st->count2;
    w.last_emitted = m;
    return build_from_pairs(m, nc, clamp, pack, out, w, s, post);
}

// binary search in the sorted row of v for u; mirror weight or -1
__device__ __forceinline__ int find_arc(const int *rp, const int2 *adj, int v, int u) {
    int lo = rp[v], hi = rp[v + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = adj[mid].x;
        if (x == u) return adj[mid].y;
        if (x < u) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

// Symmetry: every arc (u, v, c) with u < v has its mirror (v, u, c), and as
// many arcs run downwards as upwards.  Rows hold no duplicates, so the
// mirror map from upward to downward arcs is injective, and equal counts
// make it a bijection.
__global__ void k_check_sym(const DevGraph g, int *err, unsigned long long *up,
                            unsigned long long *down) {
    long long nu = 0, nd = 0;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < g.arcs; j += (i64)gridDim.x * blockDim.x) {
        const int u = g.src[j];
        const int2 e = g.adj[j];
        if (u < e.x) {
            ++nu;
            if (find_arc(g.rp, g.adj, e.x, u) != e.y) atomicOr(err, kErrAsym);
        } else {
            ++nd;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        nd += __shfl_xor_sync(0xffffffffu, nd, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nu) atomicAdd(up, (unsigned long long)nu);
        if (nd) atomicAdd(down, (unsigned long long)nd);
    }
}

__global__ void k_clear_err(Status *st) {
    st->err = 0;
    st->sym_up = 0;
    st->sym_down = 0;
    st->sym_bad = 0;
}

// Raw CSR -> graph (sources, {neighbour, weight}, degrees) in one pass,
// flagging whether the input was canonical already (rows strictly
// increasing, no self-loop, weights > 0; if not, the sort path rebuilds the
// graph) and whether it is invalid (range, negative weight).  One warp per
// row.  w == nullptr: an unweighted graph, every arc of weight 1.
// With `check`, the symmetry of input that turns out canonical is checked on
// the way (rows < u are complete whenever row u is, also when the input
// arrives in chunks of rows): every downward arc (u, v, c), v < u, must find
// its mirror (v, u, c) in v's row, and as many arcs must run up as down (the
// mirror map is then a bijection).  Neighbour ids are 4 bytes here, so a
// search reads fewer sectors than in the built 8-byte arcs.
__global__ void k_build_canon(const int *__restrict__ rp, const int *__restrict__ col,
                              const int *__restrict__ w, int n, int u_lo, int u_hi, DevGraph out, int *err,
                              int *noncanon, Status *sym) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    bool bad = false, asym = false;
    long long nu = 0, nd = 0;
    for (int u = u_lo + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); u < u_hi; u += nw) {
        const int a0 = rp[u], a1 = rp[u + 1];
        long long d = 0;
        for (int i = a0 + lane; i < a1; i += 32) {
            const int v = col[i], c = w ? w[i] : 1;
            if (v < 0 || v >= n) atomicOr(err, kErrRange);
            else if (c < 0) atomicOr(err, kErrNegW);
            if (v == u || c <= 0 || (i > a0 && col[i - 1] >= v)) bad = true;
            out.src[i] = u;
            out.adj[i] = make_int2(v, c);
            d += c;
            if (sym && v >= 0 && v < n) {
                if (v > u) {
                    ++nu;
                } else if (v < u) {
                    ++nd;
                    int lo = rp[v], hi = rp[v + 1] - 1, found = -1;
                    while (lo <= hi) {
                        const int mid = (lo + hi) >> 1;
                        const int x = col[mid];
                        if (x == u) { found = mid; break; }
                        if (x < u) lo = mid + 1; else hi = mid - 1;
                    }
                    asym |= found < 0 || (w ? w[found] : 1) != c;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) out.deg[u] = d;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(noncanon, 1);
    if (sym) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nu += __shfl_xor_sync(0xffffffffu, nu, o);
            nd += __shfl_xor_sync(0xffffffffu, nd, o);
        }
        const bool any_asym = __any_sync(0xffffffffu, asym);
        if (lane == 0) {
            if (nu) atomicAdd(reinterpret_cast<unsigned long long *>(&sym->sym_up), (unsigned long long)nu);
            if (nd) atomicAdd(reinterpret_cast<unsigned long long *>(&sym->sym_down), (unsigned long long)nd);
            if (any_asym) atomicOr(&sym->sym_bad, 1);
        }
    }
}

int canonicalize(int n, const int *rp, const int *col, const int *w, bool check_sym, DevGraph &out,
                 Work &wk, cudaStream_t s, const StagedInput *staged) {
    ++::mc::g_launches; k_clear_err<<<1, 1, 0, s>>>(wk.st);
    ++::mc::g_launches; k_check_rp<<<grid_for(n), kThreads, 0, s>>>(rp, n, &wk.st->err);
    MC_TRY(status_read(wk, s));
    if (wk.h_st->err) return MC_EINVAL;
    int arcs_raw = 0;
    if (staged) {
        arcs_raw = (int)staged->arcs;
    } else {
        MC_CUDA(cudaMemcpyAsync(&arcs_raw, rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
    }
    if (arcs_raw < 0 || (i64)arcs_raw > wk.cap_arcs) return MC_EINVAL;
    // already canonical (the common case): built directly, no sort; staged
    // input chunk by chunk as it lands
    int *noncanon = reinterpret_cast<int *>(&wk.st->count2);
    Status *sym = check_sym ? wk.st : nullptr;  // zeroed with the error bits
    ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(wk.st);
    MC_CUDA(cudaMemcpyAsync(out.rp, rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
    if (staged && staged->chunks > 0) {
        for (int k = 0; k < staged->chunks; ++k) {
            MC_CUDA(cudaStreamWaitEvent(s, staged->ready[k], 0));
            const int lo = staged->row_split[k], hi = staged->row_split[k + 1];
            if (hi <= lo) continue;
            ++::mc::g_launches;
            k_build_canon<<<grid_for((i64)(hi - lo) * 32), kThreads, 0, s>>>(rp, col, w, n, lo, hi, out,
                                                                          &wk.st->err, noncanon, sym);
        }
    } else {
        ++::mc::g_launches;
        k_build_canon<<<grid_for((i64)n * 32), kThreads, 0, s>>>(rp, col, w, n, 0, n, out, &wk.st->err, noncanon,
                                                                  sym);
    }
    MC_CUDA(cudaGetLastError());
    MC_TRY(status_read(wk, s));
    if (wk.h_st->err) return MC_EINVAL;
    out.n = n;
    out.arcs = arcs_raw;
    const bool canonical_input = wk.h_st->count2 == 0;
    if (!canonical_input) {
        ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(wk.st);
        ++::mc::g_launches; k_emit_raw<<<grid_for(((i64)arcs_raw + kEmitItems - 1) / kEmitItems), kThreads, 0, s>>>(
            rp, col, w, n, arcs_raw, wk.keysA, wk.valsA, reinterpret_cast<u64 *>(&wk.st->count), &wk.st->err);
        MC_CUDA(cudaGetLastError());
        MC_TRY(status_read(wk, s));
        if (wk.h_st->err) return MC_EINVAL;
        const i64 m = wk.h_st->count;
        MC_TRY(build_from_pairs(m, n, LLONG_MAX, 0, out, wk, s, {}));
    }
    if (canonical_input) {
        // checked while it was built
        if (check_sym && (wk.h_st->sym_bad || wk.h_st->sym_up != wk.h_st->sym_down)) return MC_EINVAL;
        return MC_OK;
    }
    ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(wk.st);
    if (check_sym && out.arcs > 0) {
        auto *up = reinterpret_cast<unsigned long long *>(&wk.st->count);
        auto *down = reinterpret_cast<unsigned long long *>(&wk.st->count2);
        ++::mc::g_launches; k_check_sym<<<grid_for(out.arcs), kThreads, 0, s>>>(out, &wk.st->err, up, down);
        MC_CUDA(cudaGetLastError());
    }
    MC_TRY(status_read(wk, s));
    if (wk.h_st->err & kErrOverflow) return MC_EOVERFLOW;
    if (wk.h_st->err & kErrNoProgress) return MC_EINTERNAL;
    if (wk.h_st->err) return MC_EINVAL;
    if (check_sym && wk.h_st->count != wk.h_st->count2) return MC_EINVAL;
    return MC_OK;
}

// ------------------------------------------------- connected components ---
// Sampled union-find (the scheme of Afforest, Sutton et al. 2018): unite
// every vertex with its first kCcSample neighbours, find the most common
// root among a sample of vertices, then process all arcs of the vertices
// outside that component only.  Exact on symmetric graphs: an arc between
// the big component and a vertex w outside it is also an arc of w.
constexpr int kCcSample = 4;
constexpr int kCcProbe = 1024;

// one thread per (vertex, sampled arc)
__global__ void k_cc_sample(const DevGraph g, int *par) {
    const i64 total = (i64)g.n * kCcSample;
    for (i64 t = (i64)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (i64)gridDim.x * blockDim.x) {
        const int v = (int)(t / kCcSample), j = (int)(t % kCcSample);
        const int i = g.rp[v] + j;
        if (i < g.rp[v + 1]) uf_union(par, v, g.adj[i].x);
    }
}

// most common root among kCcProbe evenly spaced vertices -> *giant
__global__ void __launch_bounds__(kCcProbe) k_cc_giant(const int *__restrict__ root, int n, int *giant) {
    __shared__ int key[2 * kCcProbe];
    __shared__ int cnt[2 * kCcProbe];
    __shared__ unsigned long long best;
    for (int i = threadIdx.x; i < 2 * kCcProbe; i += blockDim.x) { key[i] = -1; cnt[i] = 0; }
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    const int v = (int)(((long long)threadIdx.x * n) / kCcProbe);
    const int r = root[v];
    unsigned h = ((unsigned)r * 2654435761u) & (2 * kCcProbe - 1);
    while (true) {
        const int k = atomicCAS(&key[h], -1, r);
        if (k == -1 || k == r) break;
        h = (h + 1) & (2 * kCcProbe - 1);
    }
    const int c = atomicAdd(&cnt[h], 1) + 1;
    // largest count, then smallest root
    atomicMax(&best, ((unsigned long long)c << 32) | (unsigned)(0x7FFFFFFF - r));
    __syncthreads();
    if (threadIdx.x == 0) *giant = 0x7FFFFFFF - (int)(best & 0xFFFFFFFFu);
}

__global__ void k_cc_finish(const DevGraph g, const int *__restrict__ root, const int *giant, int *par) {
    const int G = *giant;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < g.n; v += nw) {
        if (root[v] == G) continue;
        const int a0 = g.rp[v], a1 = g.rp[v + 1];
        for (int i = a0 + kCcSample + lane; i < a1; i += 32) uf_union(par, v, g.adj[i].x);
    }
}

int connected_components(const DevGraph &g, Work &w, int *ncomp, cudaStream_t s) {
    MC_TRY(union_find_init(w.par, g.n, s));
    if (g.arcs > 0) {
        int *giant = reinterpret_cast<int *>(&w.st->count2);
        ++::mc::g_launches; k_cc_sample<<<grid_for((i64)g.n * kCcSample), kThreads, 0, s>>>(g, w.par);
        ++::mc::g_launches; k_flatten<<<grid_for(g.n), kThreads, 0, s>>>(w.par, w.root, w.cnt, g.n, nullptr);
        ++::mc::g_launches; k_cc_giant<<<1, kCcProbe, 0, s>>>(w.root, g.n, giant);
        ++::mc::g_launches; k_cc_finish<<<grid_for((i64)g.n * 32), kThreads, 0, s>>>(g, w.root, giant, w.par);
    }
    ++::mc::g_launches; k_flatten<<<grid_for(g.n), kThreads, 0, s>>>(w.par, w.root, w.cnt, g.n, nullptr);
    ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(w.st);
    MC_TRY(exclusive_scan_i32(w.cnt, w.lab, g.n, reinterpret_cast<int *>(&w.st->count), w.scan_tmp, &w.st->err, s));
    MC_TRY(status_read(w, s));
    *ncomp = (int)w.h_st->count;
    return MC_OK;
}

// ------------------------------------------------------------ side bits ---
// bit v of the side bitmap, one warp per 32 vertices
template <class F>
__global__ void k_side_bits(int n0, u32 *bits, F f) {
    const int lane = threadIdx.x & 31;
    const int nw = (n0 + 31) / 32;
    for (int wd = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wd < nw; wd += (gridDim.x * blockDim.x) >> 5) {
        int v = wd * 32 + lane;
        bool b = v < n0 && f(v);
        unsigned m = __ballot_sync(0xffffffffu, b);
        if (lane == 0) bits[wd] = m;
    }
}

struct SideVertex {
    const int *orig;
    int vertex;
    __device__ bool operator()(int v) const { return orig[v] == vertex; }
};
struct SideScan {
    const int *orig, *T, *order;
    int scan, len;
    __device__ bool operator()(int v) const {
        int c = orig[v];
        return T[c] == scan && order[c] < len;
    }
};
struct SideComp {
    const int *root;
    __device__ bool operator()(int v) const { return root[v] != root[0]; }
};

static int side_grid(int n0) { return grid_for(((i64)n0 + 31) / 32 * 32); }

int side_from_vertex(Work &w, int n0, int vertex, cudaStream_t s) {
    ++::mc::g_launches; k_side_bits<<<side_grid(n0), kThreads, 0, s>>>(n0, w.best_side, SideVertex{w.orig, vertex});
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int side_from_scan(Work &w, int n0, int scan, int len, cudaStream_t s) {
    ++::mc::g_launches; k_side_bits<<<side_grid(n0), kThreads, 0, s>>>(n0, w.best_side, SideScan{w.orig, w.T, w.order, scan, len});
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int side_from_component(Work &w, int n0, cudaStream_t s) {
    ++::mc::g_launches; k_side_bits<<<side_grid(n0), kThreads, 0, s>>>(n0, w.best_side, SideComp{w.root});
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

__global__ void k_orig_update(int *orig, const int *__restrict__ lab, int n0) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n0; v += gridDim.x * blockDim.x)
        orig[v] = lab[orig[v]];
}

int orig_update(Work &w, int n0, cudaStream_t s) {
    ++::mc::g_launches; k_orig_update<<<grid_for(n0), kThreads, 0, s>>>(w.orig, w.lab, n0);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

}  // namespace mc

namespace mc {

int flatten_labels(Work &w, int n, cudaStream_t s) {
    ++::mc::g_launches; k_flatten<<<grid_for(n), kThreads, 0, s>>>(w.par, w.root, w.cnt, n, nullptr);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

__device__ __forceinline__ void round_reset_body(Status *st, long long lam) {
    st->lam = lam;
    st->unions = 0;
    st->scanned_arcs = 0;
    st->scanned_verts = 0;
    st->scans = 0;
    st->blacklisted = 0;
    st->err = 0;
}

__global__ void k_round_reset(Status *st, long long lam) { round_reset_body(st, lam); }

// union_find_init and round_reset in one launch
__global__ void k_round_start(int *par, int n, Status *st, long long lam) {
    if (blockIdx.x == 0 && threadIdx.x == 0) round_reset_body(st, lam);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) par[v] = v;
}

int round_start(Work &w, int n, i64 lam, cudaStream_t s) {
    ++::mc::g_launches; k_round_start<<<grid_for(n), kThreads, 0, s>>>(w.par, n, w.st, lam);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int round_reset(Work &w, i64 lam, cudaStream_t s) {
    ++::mc::g_launches; k_round_reset<<<1, 1, 0, s>>>(w.st, lam);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// canonical polarity: vertex 0 on side 0; clear the bits past n0
__global__ void k_side_flip(const u32 *bits, int *flip) { *flip = (int)(bits[0] & 1u); }

__global__ void k_side_canon(u32 *bits, int n0, const int *flip_p) {
    const int nw = (n0 + 31) / 32;
    const bool flip = *flip_p != 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        u32 v = flip ? ~bits[i] : bits[i];
        if (i == nw - 1 && (n0 & 31)) v &= (1u << (n0 & 31)) - 1u;
        bits[i] = v;
    }
}

int side_canon(Work &w, int n0, cudaStream_t s) {
    // vertex 0's bit is read by its own launch before any word is rewritten
    ++::mc::g_launches; k_side_flip<<<1, 1, 0, s>>>(w.best_side, &w.st->flip);
    ++::mc::g_launches; k_side_canon<<<side_grid(n0), kThreads, 0, s>>>(w.best_side, n0, &w.st->flip);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int iota_i32(int *a, int n, cudaStream_t s) {
    ++::mc::g_launches; k_iota<<<grid_for(n), kThreads, 0, s>>>(a, n);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// flatten a caller-provided union-find array: root[v] = root of v
int flatten_raw(int *par, int *root, int *cnt, int n, cudaStream_t s) {
    ++::mc::g_launches; k_flatten<<<grid_for(n), kThreads, 0, s>>>(par, root, cnt, n, nullptr);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

__global__ void k_mark_used(const int *__restrict__ lab, int *used, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) used[v] = 0;
}

__global__ void k_mark_used2(const int *__restrict__ lab, int *used, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) used[lab[v]] = 1;
}

__global__ void k_apply_ids(int *lab, const int *__restrict__ ids, int n) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) lab[v] = ids[lab[v]];
}

int compact_labels(Work &w, int n, int *nc, cudaStream_t s) {
    ++::mc::g_launches; k_mark_used<<<grid_for(n), kThreads, 0, s>>>(w.lab, w.root, n);
    ++::mc::g_launches; k_mark_used2<<<grid_for(n), kThreads, 0, s>>>(w.lab, w.root, n);
    ++::mc::g_launches; k_zero_count<<<1, 1, 0, s>>>(w.st);
    MC_TRY(exclusive_scan_i32(w.root, w.par, n, reinterpret_cast<int *>(&w.st->count), w.scan_tmp, &w.st->err, s));
    ++::mc::g_launches; k_apply_ids<<<grid_for(n), kThreads, 0, s>>>(w.lab, w.par, n);
    MC_CUDA(cudaGetLastError());
    MC_TRY(status_read(w, s));
    *nc = (int)w.h_st->count;
    return MC_OK;
}

struct SideBits {
    const int *orig;
    const u32 *bits;
    __device__ bool operator()(int v) const {
        const int c = orig[v];
        return (bits[c >> 5] >> (c & 31)) & 1u;
    }
};

int side_from_bits(Work &w, int n0, const u32 *bits, cudaStream_t s) {
    ++::mc::g_launches; k_side_bits<<<side_grid(n0), kThreads, 0, s>>>(n0, w.best_side, SideBits{w.orig, bits});
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

struct SideRank {
    const int *rank;
    const int *orig;  // original vertex -> ranked vertex, or null (identity)
    int k;
    __device__ bool operator()(int v) const { return rank[orig ? orig[v] : v] < k; }
};

int side_from_rank(Work &w, int n0, int k, bool through_orig, cudaStream_t s) {
    ++::mc::g_launches;
    k_side_bits<<<side_grid(n0), kThreads, 0, s>>>(n0, w.best_side, SideRank{w.root, through_orig ? w.orig : nullptr, k});
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

}  // namespace mc
