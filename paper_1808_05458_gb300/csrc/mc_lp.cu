// mc_lp.cu -- label propagation (VieCut's clustering, Sec. 2.3) and the
// label-propagation upper bound on lambda.
//
// The paper names the method (Raghavan et al.) but not its rule; the rule
// used here, and by the oracle, is: labels start as vertex ids; every sweep
// has two half-sweeps p = 0, 1; in half-sweep p each vertex with
// parity(seed, sweep, v) = p takes, all at once from the labels as they
// stand, the label of largest total arc weight among its neighbours (ties to
// the smallest label; a vertex without neighbours keeps its label), where
//   parity(seed, s, v) = splitmix64(seed ^ splitmix64((s << 32) | v)) & 1.
//
// Kernels: a warp takes 32 consecutive vertices at a time.  The rows of its
// active vertices (at most kLpRow arcs each) are laid end to end and cut
// into batches of whole rows holding at most kLpBatch arcs; every lane then
// gathers up to kLpBatch / 32 arcs of a batch at once -- all of their
// {neighbour, weight} loads issued together, then all of their label loads
// -- and adds each arc's weight into a per-warp shared-memory hash keyed by
// (row, label).  Each row's choice comes from one pass over the table with
// 32-bit entries (a 64-bit atomicMax of total << 27 | (2^27 - 1 - label) per
// row: the largest total, ties to the smallest label), or, with 64-bit
// entries, two: the largest total weight (32-bit shared atomics while every
// total fits in 31 bits, else one lane compares them all), then the smallest
// label reaching it.  Longer rows
// go to a block-per-vertex kernel with a global-memory hash slice of
// 2^k > deg slots.
#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr int kLpWarps = 4;         // warps per block (19 KB of shared memory, 35 KB with 64-bit entries)
constexpr int kLpRow = 256;         // longest row handled by the warp kernel
constexpr int kLpBatch = 256;       // arcs per batch (whole rows)
constexpr int kLpPer = kLpBatch / 32;
constexpr int kLpHash = 512;        // per-warp hash slots (load <= 1/2)
constexpr int kLpBigThreads = 256;

__device__ __forceinline__ int lp_parity(u64 seed, int sweep, int v) {
    return (int)(splitmix64(seed ^ splitmix64(((u64)(unsigned)sweep << 32) | (u64)(unsigned)v)) & 1ULL);
}

// better (weight, label): larger weight, then smaller label
__device__ __forceinline__ bool lp_better(long long w1, int l1, long long w2, int l2) {
    return w1 > w2 || (w1 == w2 && l1 < l2);
}

__device__ __forceinline__ void warp_argmax(long long &w, int &l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long ow = __shfl_xor_sync(0xffffffffu, w, o);
        const int ol = __shfl_xor_sync(0xffffffffu, l, o);
        if (lp_better(ow, ol, w, l)) { w = ow; l = ol; }
    }
}

// hash entries: (row << 32 | label, 64-bit total), or, when every label is
// below 2^27 and every total below 2^31 (each weighted degree is), a 32-bit
// key (row << 27 | label) and a 32-bit total: half the shared memory and
// 32-bit atomics
template <bool NARROW>
struct LpT {
    using K = unsigned long long;
    using V = unsigned long long;
    static constexpr K kEmpty = ~0ULL;
    __device__ static K key(int row, int lab) { return ((K)row << 32) | (unsigned)lab; }
    __device__ static int row(K k) { return (int)(k >> 32); }
    __device__ static int lab(K k) { return (int)(unsigned)k; }
    __device__ static unsigned slot(K k) {
        const unsigned x = (unsigned)k * 2654435761u ^ (unsigned)(k >> 32) * 0x85EBCA6Bu;
        return x >> (32 - 9);
    }
};
template <>
struct LpT<true> {
    using K = unsigned;
    using V = unsigned;
    static constexpr K kEmpty = 0xFFFFFFFFu;
    __device__ static K key(int row, int lab) { return ((unsigned)row << 27) | (unsigned)lab; }
    __device__ static int row(K k) { return (int)(k >> 27); }
    __device__ static int lab(K k) { return (int)(k & ((1u << 27) - 1u)); }
    __device__ static unsigned slot(K k) { return (k * 2654435761u) >> (32 - 9); }
};

template <bool NARROW>
struct LpSmem {
    typename LpT<NARROW>::K key[kLpHash];  // see LpT, or kEmpty
    typename LpT<NARROW>::V val[kLpHash];  // summed arc weight
    unsigned long long best[32];           // per row (32-bit entries): packed total and label
    unsigned bw[32];                       // per row: largest total weight (31-bit totals)
    long long wide_w[32];                  // per row: the same, when a total needs more bits
    int bl[32];                            // per row: smallest label with it
    int end[32];                           // per row: end of its arcs, laid end to end
    int a0[32];                            // per row: its first arc
};

template <bool NARROW>
__global__ void __launch_bounds__(kLpWarps * 32)
k_lp_warp(const int *__restrict__ rp, const int2 *__restrict__ adj, int n, const int *__restrict__ lin,
          int *__restrict__ lout, u64 seed, int sweep, int half, int *big_list, int *big_count) {
    static_assert(kLpHash == 512, "the slot takes 9 bits");
    using T = LpT<NARROW>;
    using K = typename T::K;
    using V = typename T::V;
    __shared__ LpSmem<NARROW> sm[kLpWarps];
    LpSmem<NARROW> &h = sm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < kLpHash; i += 32) { h.key[i] = T::kEmpty; h.val[i] = 0; }
    h.best[lane] = 0;
    h.bw[lane] = 0;
    h.wide_w[lane] = -1;
    h.bl[lane] = INT_MAX;
    __syncwarp();
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nw * 32) {
        const int v = base + lane;
        int a0 = 0, d = 0;
        if (v < n) {
            const int cur = lin[v];
            a0 = rp[v];
            d = rp[v + 1] - a0;
            const bool act = lp_parity(seed, sweep, v) == half && d > 0;
            if (act && d > kLpRow) {  // hub: the block kernel decides
                big_list[atomicAdd(big_count, 1)] = v;
                d = 0;
            } else if (!act) {
                lout[v] = cur;
                d = 0;
            }
        }
        if (!__any_sync(0xffffffffu, d > 0)) continue;
        // lay the active rows end to end (inclusive scan of their lengths)
        int e = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, e, o);
            if (lane >= o) e += t;
        }
        h.end[lane] = e;
        h.a0[lane] = a0;
        // greedy batches of whole rows with at most kLpBatch arcs each
        int batch = 0, acc = 0, my_batch = 0;
        for (int j = 0; j < 32; ++j) {
            const int dj = __shfl_sync(0xffffffffu, d, j);
            if (acc + dj > kLpBatch) { ++batch; acc = 0; }
            acc += dj;
            if (lane == j) my_batch = batch;
        }
        __syncwarp();
        for (int b = 0; b <= batch; ++b) {
            const unsigned in_b = __ballot_sync(0xffffffffu, d > 0 && my_batch == b);
            if (!in_b) continue;
            const int jlo = __ffs(in_b) - 1, jhi = 31 - __clz(in_b);
            const int p0 = jlo > 0 ? h.end[jlo - 1] : 0, p1 = h.end[jhi];
            // this lane's arcs: positions p0 + lane + 32 k of the laid-out rows
            int row[kLpPer], ai[kLpPer];
#pragma unroll
            for (int k = 0; k < kLpPer; ++k) {
                const int p = p0 + lane + 32 * k;
                row[k] = -1;
                ai[k] = 0;
                if (p < p1) {
                    int lo = jlo, hi = jhi;  // the first row whose end lies past p
                    while (lo < hi) {
                        const int mid = (lo + hi) >> 1;
                        if (h.end[mid] > p) hi = mid; else lo = mid + 1;
                    }
                    row[k] = lo;
                    ai[k] = h.a0[lo] + p - (lo > 0 ? h.end[lo - 1] : 0);
                }
            }
            int2 ed[kLpPer];
#pragma unroll
            for (int k = 0; k < kLpPer; ++k) ed[k] = row[k] >= 0 ? adj[ai[k]] : make_int2(0, 0);
            int lab[kLpPer];
#pragma unroll
            for (int k = 0; k < kLpPer; ++k) lab[k] = row[k] >= 0 ? lin[ed[k].x] : 0;
#pragma unroll
            for (int k = 0; k < kLpPer; ++k) {
                if (row[k] < 0) continue;
                const K key = T::key(row[k], lab[k]);
                unsigned sl = T::slot(key);
                while (true) {
                    const K old = atomicCAS(&h.key[sl], T::kEmpty, key);
                    if (old == T::kEmpty || old == key) break;
                    sl = (sl + 1) & (kLpHash - 1);
                }
                atomicAdd(&h.val[sl], (V)ed[k].y);
            }
            __syncwarp();
            if constexpr (NARROW) {
                // one pass: per row the largest (total, smallest label) as a
                // 58-bit word (total << 27 | (2^27 - 1 - label)) by a shared
                // 64-bit atomicMax; empty the table
                for (int i = lane; i < kLpHash; i += 32) {
                    const K key = h.key[i];
                    if (key != T::kEmpty) {
                        const unsigned long long pk =
                            ((unsigned long long)h.val[i] << 27) | (unsigned)((1 << 27) - 1 - T::lab(key));
                        atomicMax(&h.best[T::row(key)], pk);
                        h.key[i] = T::kEmpty;
                        h.val[i] = 0;
                    }
                }
                __syncwarp();
                if ((in_b >> lane) & 1u) {
                    lout[v] = (1 << 27) - 1 - (int)(h.best[lane] & ((1u << 27) - 1u));
                    h.best[lane] = 0;
                }
                __syncwarp();
                continue;
            }
            // pass 1: each row's largest total weight, by 32-bit atomics while
            // every total fits in 31 bits (else one lane compares them all)
            bool wide = false;
            for (int i = lane; i < kLpHash; i += 32) {
                const K key = h.key[i];
                if (key == T::kEmpty) continue;
                const V t = h.val[i];
                if (!NARROW && (t >> 31)) wide = true;
                else atomicMax(&h.bw[T::row(key)], (unsigned)t);
            }
            if (!NARROW && __any_sync(0xffffffffu, wide)) {
                __syncwarp();
                if (lane == 0) {
                    for (int i = 0; i < kLpHash; ++i) {
                        const K key = h.key[i];
                        if (key == T::kEmpty) continue;
                        const int r = T::row(key);
                        const int l = T::lab(key);
                        if (lp_better((long long)h.val[i], l, h.wide_w[r], h.bl[r])) {
                            h.wide_w[r] = (long long)h.val[i];
                            h.bl[r] = l;
                        }
                        h.key[i] = T::kEmpty;
                        h.val[i] = 0;
                    }
                }
            } else {
                __syncwarp();
                // pass 2: the smallest label reaching it; empty the table
                for (int i = lane; i < kLpHash; i += 32) {
                    const K key = h.key[i];
                    if (key != T::kEmpty) {
                        const int r = T::row(key);
                        if (h.val[i] == (V)h.bw[r]) atomicMin(&h.bl[r], T::lab(key));
                        h.key[i] = T::kEmpty;
                        h.val[i] = 0;
                    }
                }
            }
            __syncwarp();
            if ((in_b >> lane) & 1u) {
                lout[v] = h.bl[lane];
                h.bw[lane] = 0;
                h.wide_w[lane] = -1;
                h.bl[lane] = INT_MAX;
            }
            __syncwarp();
        }
    }
}

// one block per hub vertex; a hash slice of 2^cap_log2 slots per block at
// hash_key/hash_val, of which a row of d arcs uses the smallest power of two
// >= 2d (load at most 1/2)
__global__ void __launch_bounds__(kLpBigThreads)
k_lp_big(const int *__restrict__ rp, const int2 *__restrict__ adj, const int *__restrict__ lin,
         int *__restrict__ lout, const int *__restrict__ big_list, const int *big_count,
         int *hash_key, unsigned long long *hash_val, int cap_log2) {
    __shared__ long long sw[kLpBigThreads / 32];
    __shared__ int sl[kLpBigThreads / 32];
    for (int b = blockIdx.x; b < *big_count; b += gridDim.x) {
        const int v = big_list[b];
        int *hk = hash_key + ((size_t)blockIdx.x << cap_log2);
        unsigned long long *hv = hash_val + ((size_t)blockIdx.x << cap_log2);
        const int d = rp[v + 1] - rp[v];
        int cap = 2;
        while (cap < 2 * d && cap < (1 << cap_log2)) cap <<= 1;
        for (int i = threadIdx.x; i < cap; i += blockDim.x) { hk[i] = -1; hv[i] = 0; }
        __syncthreads();
        for (int i = rp[v] + threadIdx.x; i < rp[v + 1]; i += blockDim.x) {
            const int2 e = adj[i];
            const int lab = lin[e.x];
            unsigned hh = ((unsigned)lab * 2654435761u) & (unsigned)(cap - 1);
            while (true) {
                const int k = atomicCAS(&hk[hh], -1, lab);
                if (k == -1 || k == lab) break;
                hh = (hh + 1) & (unsigned)(cap - 1);
            }
            atomicAdd(&hv[hh], (unsigned long long)e.y);
        }
        __syncthreads();
        long long bw = -1;
        int bl = INT_MAX;
        for (int i = threadIdx.x; i < cap; i += blockDim.x) {
            const int k = hk[i];
            if (k >= 0 && lp_better((long long)hv[i], k, bw, bl)) { bw = (long long)hv[i]; bl = k; }
        }
        warp_argmax(bw, bl);
        if ((threadIdx.x & 31) == 0) { sw[threadIdx.x >> 5] = bw; sl[threadIdx.x >> 5] = bl; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < kLpBigThreads / 32; ++k)
                if (lp_better(sw[k], sl[k], bw, bl)) { bw = sw[k]; bl = sl[k]; }
            lout[v] = bl;
        }
        __syncthreads();
    }
}

// longest row (*out) and largest weighted degree (*out_deg)
__global__ void k_max_row(const int *__restrict__ rp, const i64 *__restrict__ deg, int n, int *out,
                          unsigned long long *out_deg) {
    int best = 0;
    long long bd = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        best = max(best, rp[v + 1] - rp[v]);
        bd = max(bd, (long long)deg[v]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        bd = max(bd, __shfl_xor_sync(0xffffffffu, bd, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, best);
        atomicMax(out_deg, (unsigned long long)bd);
    }
}

}  // namespace

// `iters` sweeps of label propagation on g; labels (device int32[n]) hold the
// result.  Uses w.cnt as the second label buffer, w.T as the hub list and the
// radix buffers as the hubs' hash.
int label_prop(const DevGraph &g, Work &w, int iters, u64 seed, int *labels, cudaStream_t s) {
    const int n = g.n;
    MC_TRY(iota_i32(labels, n, s));
    if (iters <= 0 || n == 0) return MC_OK;
    int *d_cnt = reinterpret_cast<int *>(&w.st->count);      // hubs this half-sweep
    int *d_max = reinterpret_cast<int *>(&w.st->count2);     // longest row
    MC_CUDA(cudaMemsetAsync(&w.st->count, 0, 2 * sizeof(long long), s));
    int blocks_v = (n + 255) / 256;
    if (blocks_v > num_sms() * 8) blocks_v = num_sms() * 8;
    ++::mc::g_launches;
    k_max_row<<<blocks_v, 256, 0, s>>>(g.rp, g.deg, n, d_max, reinterpret_cast<unsigned long long *>(&w.st->count));
    MC_TRY(status_read(w, s));
    const int maxrow = (int)w.h_st->count2;
    // 32-bit hash entries: labels < 2^27, and a row's total per label is at
    // most its weighted degree
    const bool narrow = n < (1 << 27) && w.h_st->count < (1LL << 31);
    // hub hash slices: 2^k >= twice the longest row slots each (an empty
    // slot always ends a probe), as many slices as fit in one radix buffer
    // (u64 weights in the key buffer, int keys in the value buffer)
    int cap_log2 = 1;
    while ((1 << cap_log2) < 2 * maxrow) ++cap_log2;
    // a row holding most of the graph's arcs: slices of 2^k > maxrow slots
    // (still an empty slot in every probe)
    if (((size_t)w.cap_arcs >> cap_log2) < 1 && (1 << (cap_log2 - 1)) > maxrow) --cap_log2;
    const bool hubs = maxrow > kLpRow;
    size_t hub_blocks = (size_t)w.cap_arcs >> cap_log2;
    if (hub_blocks > (size_t)num_sms() * 8) hub_blocks = (size_t)num_sms() * 8;
    if (hubs && hub_blocks < 1) {
        set_error_detail("label propagation: hub rows too long for the hash workspace");
        return MC_ENOMEM;
    }
    int *cur = labels, *nxt = w.cnt;
    // as many blocks as stay resident (the narrow kernel fits about twice as many)
    int per_sm = 0;
    if (narrow) MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lp_warp<true>, kLpWarps * 32, 0));
    else MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lp_warp<false>, kLpWarps * 32, 0));
    const int grid = num_sms() * (per_sm > 0 ? per_sm : 1);
    for (int it = 0; it < iters; ++it) {
        for (int half = 0; half < 2; ++half) {
            MC_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
            ++::mc::g_launches;
            if (narrow)
                k_lp_warp<true><<<grid, kLpWarps * 32, 0, s>>>(g.rp, g.adj, n, cur, nxt, seed, it, half, w.T, d_cnt);
            else
                k_lp_warp<false><<<grid, kLpWarps * 32, 0, s>>>(g.rp, g.adj, n, cur, nxt, seed, it, half, w.T, d_cnt);
            if (hubs) {
                ++::mc::g_launches;
                k_lp_big<<<(int)hub_blocks, kLpBigThreads, 0, s>>>(g.rp, g.adj, cur, nxt, w.T, d_cnt,
                                                                    w.valsA, w.keysA, cap_log2);
            }
            MC_CUDA(cudaGetLastError());
            int *t = cur; cur = nxt; nxt = t;
        }
    }
    if (cur != labels)
        MC_CUDA(cudaMemcpyAsync(labels, cur, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s));
    return MC_OK;
}

}  // namespace mc
