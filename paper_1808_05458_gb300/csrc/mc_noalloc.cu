// mc_noalloc.cu -- a full CAPFOREST scan that allocates no device memory.
//
// Some callers cannot allocate device memory once they are running: code
// with a rule against allocation after start-up (latency-critical or
// certified services, where cudaMalloc may synchronise the device or fail
// on a fragmented heap), or a process whose device memory is already held by
// another allocator, such as a framework's caching allocator, so that a
// fresh cudaMalloc could run out of memory.  For them, this entry point runs
// the same full-scan kernel as mc_step_capforest_full with all of its
// scratch in one file-scope device array below, which every GPU that loads
// the library holds until the process exits.  The caller passes its inputs
// and outputs; nothing is allocated per call.
//
// Set-up: the first call on a device looks up the device address of the
// array with cudaGetSymbolAddress (with that device current) and keeps it;
// make that first call before any stream capture.  Every call on a device
// shares the one array and leaves its contents behind; each call clears what
// must start at zero.  Calls whose work overlaps on the GPU (another thread,
// another stream) race on the array and must be serialised by the caller.
#include <mutex>

#include "mc_internal.cuh"

namespace mc {

namespace {

constexpr size_t kNaAlign = 256;
constexpr size_t round_up(size_t x) { return (x + kNaAlign - 1) / kNaAlign * kNaAlign; }

// scratch layout (byte offsets into the array)
constexpr size_t kNaStatus = 0;
constexpr size_t kNaPar = kNaStatus + round_up(sizeof(Status));
constexpr size_t kNaT = kNaPar + round_up(sizeof(int) * MC_NOALLOC_MAX_N);
constexpr size_t kNaOrder = kNaT + round_up(sizeof(int) * MC_NOALLOC_MAX_N);
constexpr size_t kNaR = kNaOrder + round_up(sizeof(int) * MC_NOALLOC_MAX_N);
constexpr size_t kNaCnt = kNaR + round_up(sizeof(int) * MC_NOALLOC_MAX_N);
constexpr size_t kNaDeg = kNaCnt + round_up(sizeof(int) * MC_NOALLOC_MAX_N);
constexpr size_t kNaRecA = kNaDeg + round_up(sizeof(long long) * MC_NOALLOC_MAX_N);
constexpr size_t kNaRecL = kNaRecA + round_up(sizeof(long long) * 2);
constexpr size_t kNaPool = (size_t)MC_NOALLOC_MAX_ARCS + 2;
constexpr size_t kNaSlot = kNaRecL + round_up(sizeof(int) * 2);
constexpr size_t kNaNext = kNaSlot + round_up(sizeof(int) * kNaPool);
constexpr size_t kNaBlkWords = (size_t)(kBlkMaxCap + 1) * (MC_NOALLOC_MAX_N / 32 + MC_NOALLOC_MAX_N / 1024);
constexpr size_t kNaBlk = kNaNext + round_up(sizeof(int) * kNaPool);
constexpr size_t kNaBytes = kNaBlk + round_up(sizeof(u32) * kNaBlkWords);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Input checks before any access that the input indexes: one block resets
// the status block, then checks the row offsets (row_ptr[0] = 0,
// non-decreasing, row_ptr[n] = arcs); a bad offset sets kErrRange.
__global__ void __launch_bounds__(1024) k_na_check_rp(int n, long long arcs, const int *__restrict__ rp,
                                                     long long lam) {
    Status *st = reinterpret_cast<Status *>(g_noalloc_scratch + kNaStatus);
    if (threadIdx.x == 0) {
        st->lam = lam;
        st->unions = 0;
        st->scanned_arcs = 0;
        st->scanned_verts = 0;
        st->scans = 0;
        st->blacklisted = 0;
        st->err = 0;
        st->scan_ids = 0;
        st->cursor = 0;
    }
    __syncthreads();
    bool bad = false;
    for (int v = threadIdx.x; v <= n; v += blockDim.x) {
        const int a = rp[v];
        if (v == 0 && a != 0) bad = true;
        if (v == n && (long long)a != arcs) bad = true;
        if (v < n && rp[v + 1] < a) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) st->err |= kErrRange;
}

// One warp per row, only once the offsets passed: checks every arc
// (neighbour in [0, n), not the row's own vertex, weight >= 1), sums the
// weighted degree and zeroes the row's scan state.  A bad arc sets kErrRange
// and nothing downstream runs.
__global__ void __launch_bounds__(256) k_na_prepare(int n, const int *__restrict__ rp,
                                                    const int2 *__restrict__ adj) {
    Status *st = reinterpret_cast<Status *>(g_noalloc_scratch + kNaStatus);
    if (*(volatile int *)&st->err) return;
    int *T = reinterpret_cast<int *>(g_noalloc_scratch + kNaT);
    int *r = reinterpret_cast<int *>(g_noalloc_scratch + kNaR);
    long long *deg = reinterpret_cast<long long *>(g_noalloc_scratch + kNaDeg);
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (int v = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n; v += warps) {
        const int a0 = rp[v], a1 = rp[v + 1];
        long long d = 0;
        for (int a = a0 + lane; a < a1; a += 32) {
            const int2 e = adj[a];
            if (e.x < 0 || e.x >= n || e.x == v || e.y < 1) bad = true;
            d += e.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) {
            deg[v] = d;
            T[v] = 0;
            r[v] = 0;
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&st->err, kErrRange);
}

std::mutex g_na_mutex;
void *g_na_ptr[64] = {nullptr};

// device address of the scratch array on the current device (looked up once)
int na_scratch(unsigned char **out) {
    int dev = 0;
    MC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MC_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        MC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_na_ptr[dev]);
    return MC_OK;
}

}  // namespace
}  // namespace mc

using namespace mc;

extern "C" int mc_capforest_full_noalloc(int32_t n, int64_t arcs, const int32_t *row_ptr,
                                         const int32_t *adj, int64_t lam, int32_t start,
                                         int32_t *labels, int64_t *lam_out, int64_t *unions_out,
                                         void *cuda_stream) {
    if (n < 1 || arcs < 0 || !row_ptr || !labels || start < 0 || start >= n) return MC_EINVAL;
    if (arcs > 0 && !adj) return MC_EINVAL;
    if (n > MC_NOALLOC_MAX_N || arcs > MC_NOALLOC_MAX_ARCS) {
        set_error_detail("mc_capforest_full_noalloc: graph exceeds the static scratch "
                         "(MC_NOALLOC_MAX_N vertices, MC_NOALLOC_MAX_ARCS arcs)");
        return MC_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(adj) % 8 != 0) return MC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned char *base = nullptr;
    MC_TRY(na_scratch(&base));
    Status *st = reinterpret_cast<Status *>(base + kNaStatus);

    DevGraph g;
    g.n = n;
    g.arcs = arcs;
    g.rp = const_cast<int *>(row_ptr);
    g.src = nullptr;
    g.adj = reinterpret_cast<int2 *>(const_cast<int32_t *>(adj));
    g.deg = reinterpret_cast<i64 *>(base + kNaDeg);

    ++::mc::g_launches; k_na_check_rp<<<1, 1024, 0, s>>>(n, arcs, row_ptr, lam);
    MC_CUDA(cudaGetLastError());
    int blocks = (n + 7) / 8;
    if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
    ++::mc::g_launches; k_na_prepare<<<blocks, 256, 0, s>>>(n, row_ptr, g.adj);
    MC_CUDA(cudaGetLastError());
    {
        int err = 0;
        MC_CUDA(cudaMemcpyAsync(&err, &st->err, sizeof(int), cudaMemcpyDeviceToHost, s));
        MC_CUDA(cudaStreamSynchronize(s));
        if (err) {
            set_error_detail("mc_capforest_full_noalloc: bad row offsets, or an arc with a neighbour "
                             "out of range, a self-loop or a weight below 1");
            return MC_EINVAL;
        }
    }
    int *par = reinterpret_cast<int *>(base + kNaPar);
    MC_TRY(iota_i32(par, n, s));
    MC_TRY(capforest_full_raw(g, par, reinterpret_cast<int *>(base + kNaT),
                              reinterpret_cast<int *>(base + kNaOrder), st,
                              reinterpret_cast<i64 *>(base + kNaRecA),
                              reinterpret_cast<int *>(base + kNaRecL),
                              reinterpret_cast<int *>(base + kNaR),
                              reinterpret_cast<int *>(base + kNaSlot),
                              reinterpret_cast<int *>(base + kNaNext), (int)(arcs + 2),
                              reinterpret_cast<u32 *>(base + kNaBlk), kNaBlkWords, start, s));
    MC_TRY(flatten_raw(par, labels, reinterpret_cast<int *>(base + kNaCnt), n, s));
    Status h;
    MC_CUDA(cudaMemcpyAsync(&h, st, sizeof(Status), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    if (lam_out) *lam_out = h.lam;
    if (unions_out) *unions_out = h.unions;
    return MC_OK;
}
