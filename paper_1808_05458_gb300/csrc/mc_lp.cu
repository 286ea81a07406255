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
// Kernels: one warp per vertex.  Rows of <= 32 arcs sum equal labels across
// the warp's registers; rows of <= kLpSmemRow arcs aggregate in a
// per-warp shared-memory hash; longer rows are left to a block-per-vertex
// kernel that aggregates in a global-memory hash slice of 2^k > deg slots.
#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr int kLpWarps = 4;         // warps per block
constexpr int kLpHash = 1024;       // per-warp hash slots
constexpr int kLpSmemRow = 512;     // longest row handled by the warp kernel
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

struct LpSmem {
    int key[kLpHash];
    unsigned long long val[kLpHash];
    unsigned long long sum[32];  // per-lane label weights of a short row
    short used[kLpSmemRow];      // hash slots a longer row filled
    int nused;
};

// Each warp takes 32 consecutive vertices at a time: their parities and row
// bounds come in one coalesced step, vertices outside this half-sweep keep
// their label, and the warp then works through the active ones.  A row of
// <= 32 arcs groups equal labels with match_any and adds each group's
// weights in shared memory at its lowest lane.
__global__ void __launch_bounds__(kLpWarps * 32)
k_lp_warp(const int *__restrict__ rp, const int2 *__restrict__ adj, int n, const int *__restrict__ lin,
          int *__restrict__ lout, u64 seed, int sweep, int half, int *big_list, int *big_count) {
    __shared__ LpSmem sm[kLpWarps];
    LpSmem &h = sm[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    for (int i = lane; i < kLpHash; i += 32) { h.key[i] = -1; h.val[i] = 0; }
    h.sum[lane] = 0;
    if (lane == 0) h.nused = 0;
    __syncwarp();
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nw * 32) {
        const int v = base + lane;
        int a0 = 0, a1 = 0, cur = 0;
        bool act = false;
        if (v < n) {
            cur = lin[v];
            a0 = rp[v];
            a1 = rp[v + 1];
            act = lp_parity(seed, sweep, v) == half && a1 > a0;
            if (act && a1 - a0 > kLpSmemRow) {  // hub: the block kernel decides
                big_list[atomicAdd(big_count, 1)] = v;
                act = false;
            } else if (!act) {
                lout[v] = cur;
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, act);
        while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const int u = base + l;
            const int r0 = __shfl_sync(0xffffffffu, a0, l), r1 = __shfl_sync(0xffffffffu, a1, l);
            const int d = r1 - r0;
            long long bw = -1;
            int bl = INT_MAX;
            if (d <= 32) {
                int lab = -1 - lane;
                int wt = 0;
                if (lane < d) {
                    const int2 e = adj[r0 + lane];
                    lab = lin[e.x];
                    wt = e.y;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, lab);
                const int lead = __ffs(peers) - 1;
                if (lane < d) atomicAdd(&h.sum[lead], (unsigned long long)wt);
                __syncwarp();
                if (lane < d && lead == lane) { bw = (long long)h.sum[lane]; bl = lab; }
                __syncwarp();
                h.sum[lane] = 0;
            } else {
                for (int i = r0 + lane; i < r1; i += 32) {
                    const int2 e = adj[i];
                    const int lab = lin[e.x];
                    unsigned hh = ((unsigned)lab * 2654435761u) >> (32 - 10);
                    while (true) {
                        const int k = atomicCAS(&h.key[hh], -1, lab);
                        if (k == -1) { h.used[atomicAdd(&h.nused, 1)] = (short)hh; break; }
                        if (k == lab) break;
                        hh = (hh + 1) & (kLpHash - 1);
                    }
                    atomicAdd(&h.val[hh], (unsigned long long)e.y);
                }
                __syncwarp();
                // the row's labels sit in the slots it filled (<= d of them);
                // read them, then clear exactly those
                const int nu = h.nused;
                for (int i = lane; i < nu; i += 32) {
                    const int slot = h.used[i];
                    const int k = h.key[slot];
                    if (lp_better((long long)h.val[slot], k, bw, bl)) { bw = (long long)h.val[slot]; bl = k; }
                }
                __syncwarp();
                for (int i = lane; i < nu; i += 32) {
                    const int slot = h.used[i];
                    h.key[slot] = -1;
                    h.val[slot] = 0;
                }
                if (lane == 0) h.nused = 0;
                __syncwarp();
            }
            warp_argmax(bw, bl);
            if (lane == 0) lout[u] = bl;
        }
    }
}

// one block per hub vertex; hash slice of `cap` slots at hash_key/hash_val
__global__ void __launch_bounds__(kLpBigThreads)
k_lp_big(const int *__restrict__ rp, const int2 *__restrict__ adj, const int *__restrict__ lin,
         int *__restrict__ lout, const int *__restrict__ big_list, const int *big_count,
         int *hash_key, unsigned long long *hash_val, int cap_log2) {
    const int cap = 1 << cap_log2;
    __shared__ long long sw[kLpBigThreads / 32];
    __shared__ int sl[kLpBigThreads / 32];
    for (int b = blockIdx.x; b < *big_count; b += gridDim.x) {
        const int v = big_list[b];
        int *hk = hash_key + (size_t)blockIdx.x * cap;
        unsigned long long *hv = hash_val + (size_t)blockIdx.x * cap;
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

__global__ void k_max_row(const int *__restrict__ rp, int n, int *out) {
    int best = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        best = max(best, rp[v + 1] - rp[v]);
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, best);
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
    MC_CUDA(cudaMemsetAsync(&w.st->count2, 0, sizeof(long long), s));
    int blocks_v = (n + 255) / 256;
    if (blocks_v > num_sms() * 8) blocks_v = num_sms() * 8;
    ++::mc::g_launches; k_max_row<<<blocks_v, 256, 0, s>>>(g.rp, n, d_max);
    MC_TRY(status_read(w, s));
    const int maxrow = (int)w.h_st->count2;
    // hub hash slices: 2^k > longest row slots each (an empty slot always
    // ends a probe), as many slices as fit in one radix buffer (u64 weights
    // in the key buffer, int keys in the value buffer)
    int cap_log2 = 1;
    while ((1 << cap_log2) <= maxrow) ++cap_log2;
    const bool hubs = maxrow > kLpSmemRow;
    size_t hub_blocks = (size_t)w.cap_arcs >> cap_log2;
    if (hub_blocks > 256) hub_blocks = 256;
    if (hubs && hub_blocks < 1) {
        set_error_detail("label propagation: hub rows too long for the hash workspace");
        return MC_ENOMEM;
    }
    int *cur = labels, *nxt = w.cnt;
    int grid = num_sms() * 8;
    for (int it = 0; it < iters; ++it) {
        for (int half = 0; half < 2; ++half) {
            MC_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int), s));
            ++::mc::g_launches;
            k_lp_warp<<<grid, kLpWarps * 32, 0, s>>>(g.rp, g.adj, n, cur, nxt, seed, it, half, w.T, d_cnt);
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
