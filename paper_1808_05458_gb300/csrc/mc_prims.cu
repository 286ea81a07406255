// mc_prims.cu -- errors, allocation, device-wide scan and LSD radix sort.
//
// The radix sort and scan are the building blocks of the CSR rebuild by
// "radix sort plus segmented sum" that replaces the paper's concurrent hash
// table in parallel graph contraction (Sec. 3.2).
#include <atomic>
#include <cstdio>
#include <cstring>

#include "mc_internal.cuh"
#include "mc_sort.cuh"

namespace mc {

thread_local long long g_launches = 0;

// ----------------------------------------------------------------- errors --
static thread_local std::string g_detail;

void set_cuda_error(cudaError_t e, const char *what) {
    g_detail = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e) + " in " + what;
}
void set_error_detail(const char *msg) { g_detail = msg; }
const std::string &error_detail() { return g_detail; }

// ------------------------------------------------------------- allocation --
// Stream-ordered allocations from the device's default pool, which keeps
// freed memory for reuse (release threshold raised once per device): graphs
// created and destroyed in a loop then allocate without device-wide syncs.
static void retain_pool_memory() {
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
    done[dev] = true;
}

// fault-injection hook (mc_test_fail_alloc_after): allocations to pass
// before one fails; -1 = off
static std::atomic<long long> g_fail_alloc_after{-1};

void test_fail_alloc_after(long long k) { g_fail_alloc_after.store(k < 0 ? -1 : k); }
bool test_alloc_hook_armed() { return g_fail_alloc_after.load() >= 0; }

int dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    long long k = g_fail_alloc_after.load();
    while (k >= 0 && !g_fail_alloc_after.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 0) {
        *p = nullptr;
        set_error_detail("injected allocation failure");
        return MC_ENOMEM;
    }
    retain_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        set_cuda_error(e, "cudaMallocAsync");
        return e == cudaErrorMemoryAllocation ? MC_ENOMEM : MC_ECUDA;
    }
    return MC_OK;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

int num_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

int status_read(Work &w, cudaStream_t s) {
    MC_CUDA(cudaMemcpyAsync(w.h_st, w.st, sizeof(Status), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    return MC_OK;
}

// ------------------------------------------------------------------- scan --
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// exclusive scan across the block; the block total goes to *total (a shared
// variable of the caller, valid after the call)
template <class T, int NT>
__device__ __forceinline__ T block_excl_scan(T v, T *total) {
    __shared__ T wsum[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T x = lane < NT / 32 ? wsum[lane] : T(0);
        T xs = warp_incl_scan(x);
        if (lane < NT / 32) wsum[lane] = xs - x;
        if (lane == NT / 32 - 1) *total = xs;
    }
    __syncthreads();
    T r = wsum[wid] + inc - v;
    __syncthreads();
    return r;
}

// Single-pass exclusive scan with decoupled look-back (Merrill and Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016), for up
// to kScanLookTiles tiles: each block takes the next tile index from a
// counter (so every tile it waits on belongs to a block that started before
// it), publishes its tile's sum, then reads its predecessors' published
// words, 32 * kScanLook per round trip, adding sums back to the nearest
// published prefix, and publishes its own prefix.
//
// tmp: a header {tile counter, finished blocks, epoch, -} and one 64-bit word
// per tile, (epoch << 34) | (state << 32) | value with state 1 = the tile's
// sum, 2 = its inclusive prefix; a word of another epoch is unpublished.  The
// last block to finish resets the counters and advances the epoch, so the
// buffer needs no clearing between calls (stream-ordered calls only).  A wait
// that outlasts kScanSpinLimit polls sets kErrNoProgress in *err and takes 0
// for the rest (it cannot happen while blocks start in tile order).
constexpr long long kScanSpinLimit = 1LL << 22;
constexpr int kScanLook = 8;        // predecessor words per lane and round trip
constexpr int kScanLookTiles = 256;  // larger inputs take the two-launch path

struct ScanHeader {
    unsigned tiles, done, epoch, large_done;
};

__device__ __forceinline__ u64 scan_word(unsigned epoch, unsigned state, unsigned v) {
    return ((u64)(epoch & 0x3FFFFFFFu) << 34) | ((u64)state << 32) | v;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan1(const int *in, int *out, i64 n, int *d_total, unsigned *tmp, int nt, int *err) {
    ScanHeader *hdr = reinterpret_cast<ScanHeader *>(tmp);
    u64 *words = reinterpret_cast<u64 *>(tmp + 4);
    __shared__ int s_tile, s_prefix, s_tot;
    __shared__ unsigned s_epoch;
    if (threadIdx.x == 0) {
        s_epoch = *(volatile unsigned *)&hdr->epoch;
        s_tile = (int)atomicAdd(&hdr->tiles, 1u);
    }
    __syncthreads();
    const int t = s_tile;
    const unsigned ep = s_epoch & 0x3FFFFFFFu;
    // blocked arrangement: thread k owns items [k*ITEMS, k*ITEMS+ITEMS)
    const i64 base = (i64)t * kScanTile + (i64)threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const i64 i = base + k;
        v[k] = i < n ? in[i] : 0;
        sum += v[k];
    }
    int ex = block_excl_scan<int, kScanThreads>(sum, &s_tot);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int agg = s_tot;
        if (lane == 0) *(volatile u64 *)&words[t] = scan_word(ep, t == 0 ? 2u : 1u, (unsigned)agg);
        int excl = 0;
        long long spins = 0;
        for (int j = t - 1; j >= 0;) {
            // lane l reads tiles j - l - 32k; below tile 0: a prefix of 0
            unsigned st[kScanLook], val[kScanLook];
#pragma unroll
            for (int k = 0; k < kScanLook; ++k) {
                const int idx = j - lane - 32 * k;
                st[k] = 2u;
                val[k] = 0u;
                if (idx >= 0) {
                    const u64 w = *(volatile u64 *)&words[idx];
                    st[k] = (unsigned)(w >> 34) == ep ? (unsigned)(w >> 32) & 3u : 0u;
                    val[k] = (unsigned)w;
                }
            }
            // the nearest prefix P in the window (-1: tile 0's virtual
            // predecessor, -2: none); the walk ends at P once every tile after
            // it has published
            int near = -2;
#pragma unroll
            for (int k = 0; k < kScanLook; ++k) {
                const int idx = j - lane - 32 * k;
                const int at = idx >= 0 ? idx : -1;
                if (st[k] == 2u && at > near) near = at;
            }
            const int P = __reduce_max_sync(0xffffffffu, near);
            bool waiting = false;
            unsigned part = 0;
#pragma unroll
            for (int k = 0; k < kScanLook; ++k) {
                const int idx = j - lane - 32 * k;
                if (idx >= P) {
                    waiting |= st[k] == 0u;
                    part += val[k];
                }
            }
            if (__any_sync(0xffffffffu, waiting)) {
                if (++spins > kScanSpinLimit) {
                    if (lane == 0) atomicOr(err, kErrNoProgress);
                    break;
                }
                __nanosleep(32);
                continue;
            }
            excl += (int)__reduce_add_sync(0xffffffffu, part);
            if (P >= -1) break;
            j -= 32 * kScanLook;
        }
        if (lane == 0) {
            if (t > 0) *(volatile u64 *)&words[t] = scan_word(ep, 2u, (unsigned)(excl + agg));
            s_prefix = excl;
            if (t == nt - 1 && d_total) *d_total = excl + agg;
        }
    }
    __syncthreads();
    ex += s_prefix;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const i64 i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0 && atomicAdd(&hdr->done, 1u) == (unsigned)nt - 1u) {
        // every block took its tile and finished: reset for the next call
        hdr->tiles = 0;
        hdr->done = 0;
        hdr->epoch = hdr->epoch + 1u;
    }
}

// Larger inputs: the look-back walk grows with the tile count, so two
// launches instead -- each tile's sum, the last block to finish scanning the
// sums (its counter comes back to 0), then each tile's scan from its offset.
__global__ void __launch_bounds__(kScanThreads)
k_tile_reduce(const int *__restrict__ in, i64 n, int *part, int nt, int *d_total, unsigned *done) {
    __shared__ int tot;
    __shared__ bool last;
    const i64 base = (i64)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const i64 i = base + (i64)k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    (void)block_excl_scan<int, kScanThreads>(s, &tot);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = tot;
        __threadfence();
        last = atomicAdd(done, 1u) == (unsigned)nt - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the tile sums, scanned in place by this block (a run per thread)
    const int per = (nt + kScanThreads - 1) / kScanThreads;
    const int lo = threadIdx.x * per, hi = min(nt, lo + per);
    int r = 0;
    for (int i = lo; i < hi; ++i) r += *(volatile int *)&part[i];
    int ex = block_excl_scan<int, kScanThreads>(r, &tot);
    for (int i = lo; i < hi; ++i) {
        const int v = *(volatile int *)&part[i];
        part[i] = ex;
        ex += v;
    }
    if (threadIdx.x == 0) {
        if (d_total) *d_total = tot;
        *done = 0;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_tile_scan(const int *__restrict__ in, int *__restrict__ out, i64 n, const int *__restrict__ part) {
    __shared__ int tot;
    const i64 base = (i64)blockIdx.x * kScanTile + (i64)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const i64 i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int ex = block_excl_scan<int, kScanThreads>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const i64 i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
}

// tmp: the header {tile counter, finished blocks, epoch, two-launch block
// counter}, the look-back words (2 ints per tile, at most kScanLookTiles
// tiles), then the two-launch path's tile sums (1 int per tile)
constexpr int kScanParts = 4 + 2 * kScanLookTiles;
size_t scan_tmp_words(i64 n) { return kScanParts + (size_t)div_up(n > 0 ? n : 1, kScanTile) + 32; }

int scan_tmp_clear(int *tmp, size_t words, cudaStream_t s) {
    // the look-back words too: recycled memory may hold another buffer's
    // words of the same epoch
    MC_CUDA(cudaMemsetAsync(tmp, 0, words * sizeof(int), s));
    return MC_OK;
}

int exclusive_scan_i32(const int *d_in, int *d_out, i64 n, int *d_total, int *tmp, int *err,
                       cudaStream_t s) {
    if (n <= 0) {
        if (d_total) MC_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), s));
        return MC_OK;
    }
    const int nt = div_up(n, kScanTile);
    if (nt <= kScanLookTiles) {
        ++::mc::g_launches;
        k_scan1<<<nt, kScanThreads, 0, s>>>(d_in, d_out, n, d_total, reinterpret_cast<unsigned *>(tmp), nt, err);
    } else {
        int *part = tmp + kScanParts;
        unsigned *done = reinterpret_cast<unsigned *>(tmp + 3);
        ++::mc::g_launches; k_tile_reduce<<<nt, kScanThreads, 0, s>>>(d_in, n, part, nt, d_total, done);
        ++::mc::g_launches; k_tile_scan<<<nt, kScanThreads, 0, s>>>(d_in, d_out, n, part);
    }
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// ------------------------------------------------------------- radix sort --
// LSD radix sort, 8-bit digits.  Per pass: (1) per-tile digit histograms,
// (2) one exclusive scan over the digit-major histogram matrix gives every
// (digit, tile) its output offset, (3) each tile ranks its keys stably with
// warp match/ballot, reorders them in shared memory and writes each digit's
// run contiguously.
constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // 2048
constexpr int kRsWarps = kRsThreads / 32;

__global__ void k_rs_hist(const u64 *__restrict__ keys, i64 n, int shift, int ntiles,
                          int *__restrict__ hist) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    i64 base = (i64)blockIdx.x * kRsTile;
#pragma unroll
    for (int k = 0; k < kRsItems; ++k) {
        i64 i = base + (i64)k * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(int)((keys[i] >> shift) & 255)], 1);
    }
    __syncthreads();
    hist[(i64)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// VALS: an int32 value travels with each key (else keys only)
template <bool VALS>
__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const u64 *__restrict__ kin, const int *__restrict__ vin, u64 *__restrict__ kout,
             int *__restrict__ vout, i64 n, int shift, int ntiles, const int *__restrict__ offs) {
    __shared__ u64 sk[kRsTile];
    __shared__ int sv[VALS ? kRsTile : 1];
    __shared__ int wcnt[kRsWarps][256];
    __shared__ int dstart[256];
    __shared__ int gofs[256];
    __shared__ int total;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const i64 tile0 = (i64)blockIdx.x * kRsTile;
    const int count = (int)min((i64)kRsTile, n - tile0);

#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) wcnt[wid][k * 32 + lane] = 0;
    __syncwarp();

    u64 key[kRsItems];
    int val[kRsItems], dig[kRsItems], rank[kRsItems];
    const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        int li = wid * (kRsItems * 32) + j * 32 + lane;
        i64 i = tile0 + li;
        bool ok = li < count;
        key[j] = ok ? kin[i] : ~0ULL;
        val[j] = VALS && ok ? vin[i] : 0;
        dig[j] = ok ? (int)((key[j] >> shift) & 255) : 255;
    }
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        unsigned peers = __match_any_sync(0xffffffffu, dig[j]);
        int before = __popc(peers & lt_mask);
        int base = wcnt[wid][dig[j]];
        __syncwarp();
        if (before == 0) wcnt[wid][dig[j]] = base + __popc(peers);
        __syncwarp();
        rank[j] = base + before;
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // 256 threads == 256 digits
        int run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            int c = wcnt[w][d];
            wcnt[w][d] = run;
            run += c;
        }
        int ex = block_excl_scan<int, kRsThreads>(run, &total);
        dstart[d] = ex;
        gofs[d] = offs[(i64)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRsItems; ++j) {
        int pos = dstart[dig[j]] + wcnt[wid][dig[j]] + rank[j];
        sk[pos] = key[j];
        if (VALS) sv[pos] = val[j];
    }
    __syncthreads();
    for (int p = threadIdx.x; p < count; p += kRsThreads) {
        u64 k = sk[p];
        int d = (int)((k >> shift) & 255);
        i64 o = (i64)gofs[d] + (p - dstart[d]);
        kout[o] = k;
        if (VALS) vout[o] = sv[p];
    }
}

size_t radix_tmp_words(i64 n) { return (size_t)256 * div_up(n > 0 ? n : 1, kRsTile) + 64; }

int radix_sort_pairs(u64 *keysA, int *valsA, u64 *keysB, int *valsB, i64 n, int bits, u32 *tmp,
                     int *scan_tmp, int *err, bool *in_b, cudaStream_t s) {
    *in_b = false;
    if (n <= 1 || bits <= 0) return MC_OK;
    const int ntiles = div_up(n, kRsTile);
    int *hist = reinterpret_cast<int *>(tmp);
    u64 *ki = keysA, *ko = keysB;
    int *vi = valsA, *vo = valsB;
    for (int shift = 0; shift < bits; shift += 8) {
        ++::mc::g_launches; k_rs_hist<<<ntiles, kRsThreads, 0, s>>>(ki, n, shift, ntiles, hist);
        MC_TRY(exclusive_scan_i32(hist, hist, (i64)256 * ntiles, nullptr, scan_tmp, err, s));
        ++::mc::g_launches; k_rs_scatter<true><<<ntiles, kRsThreads, 0, s>>>(ki, vi, ko, vo, n, shift, ntiles, hist);
        MC_CUDA(cudaGetLastError());
        u64 *tk = ki; ki = ko; ko = tk;
        int *tv = vi; vi = vo; vo = tv;
        *in_b = !*in_b;
    }
    return MC_OK;
}

int radix_sort_keys(u64 *keysA, u64 *keysB, i64 n, int shift0, int bits, u32 *tmp, int *scan_tmp, int *err,
                    bool *in_b, cudaStream_t s) {
    *in_b = false;
    if (n <= 1 || bits <= 0) return MC_OK;
    const int ntiles = div_up(n, kRsTile);
    int *hist = reinterpret_cast<int *>(tmp);
    u64 *ki = keysA, *ko = keysB;
    for (int shift = shift0; shift < shift0 + bits; shift += 8) {
        ++::mc::g_launches; k_rs_hist<<<ntiles, kRsThreads, 0, s>>>(ki, n, shift, ntiles, hist);
        MC_TRY(exclusive_scan_i32(hist, hist, (i64)256 * ntiles, nullptr, scan_tmp, err, s));
        ++::mc::g_launches; k_rs_scatter<false><<<ntiles, kRsThreads, 0, s>>>(ki, nullptr, ko, nullptr, n, shift,
                                                                            ntiles, hist);
        MC_CUDA(cudaGetLastError());
        u64 *tk = ki; ki = ko; ko = tk;
        *in_b = !*in_b;
    }
    return MC_OK;
}

}  // namespace mc
