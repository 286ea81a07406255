// mc_pr.cu -- Padberg-Rinaldi local contraction tests.
//
// The paper cites the tests (Sec. 2.2 related work; used by VieCut,
// Sec. 2.3) without stating them.  With d() the weighted degree of the
// current graph and lam the current bound lambda-hat (always <= delta),
// edge {u, v} of weight c is united when
//   PR1: c >= lam
//   PR2: 2c > min(d(u), d(v))
//   PR3: a common neighbour w has 2(c + c(u,w)) > d(u) and 2(c + c(v,w)) > d(v)
//   PR4: c + sum over common neighbours w of min(c(u,w), c(v,w)) >= lam
// PR1 and PR4 bound lambda(G, u, v) from below by lam (an edge and
// edge-disjoint two-edge paths).  PR2 and PR3 show that any cut below
// delta that separates u and v could be made strictly lighter by moving u
// or v across, so no minimum cut below lambda-hat crosses the edge; the
// strict inequality is what lets all passing edges be contracted at once.
// With level >= 2 a vertex with exactly two neighbours joined by equal
// weights also joins the smaller neighbour: a cut below delta crosses a path
// of such vertices at most once and slides along it at equal weight, and a
// path's k inner vertices close at most k of its k+1 edges.
//
// PR1/PR2: one thread per arc (u < v).  PR3/PR4: one warp per vertex (see
// k_pr34), only on edges whose shorter row has at most `budget` arcs (all
// edges when budget < 0).
#include "mc_internal.cuh"

namespace mc {

__device__ __forceinline__ int row_weight(const int *rp, const int2 *adj, int v, int u) {
    int lo = rp[v], hi = rp[v + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = adj[mid].x;
        if (x == u) return adj[mid].y;
        if (x < u) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

// PR1/PR2 (lo <= 2) on every arc u < v, and the degree-2 tie rule
__global__ void k_pr(const DevGraph g, int *par, long long lam, int lo, int level,
                     unsigned long long *unions) {
    long long local = 0;
    for (i64 j = (i64)blockIdx.x * blockDim.x + threadIdx.x; j < g.arcs; j += (i64)gridDim.x * blockDim.x) {
        const int u = g.src[j];
        const int2 e = g.adj[j];
        const int v = e.x;
        if (u >= v) continue;
        const long long c = e.y;
        const long long du = g.deg[u], dv = g.deg[v];
        bool ok = (lo <= 1 && level >= 1 && c >= lam) ||
                  (lo <= 2 && level >= 2 && 2 * c > (du < dv ? du : dv));
        if (ok && uf_union(par, u, v)) ++local;
    }
    // degree-2 tie rule: a vertex with exactly two neighbours of equal weight
    // joins the smaller one (a cut below delta slides along such a path)
    if (lo <= 2 && level >= 2) {
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < g.n; u += gridDim.x * blockDim.x) {
            const int a = g.rp[u];
            if (g.rp[u + 1] - a != 2) continue;
            const int2 e0 = g.adj[a], e1 = g.adj[a + 1];
            if (e0.y == e1.y && uf_union(par, u, e0.x < e1.x ? e0.x : e1.x)) ++local;
        }
    }
    if (local) atomicAdd(unions, (unsigned long long)local);
}

// PR3/PR4, one warp per vertex u.  Edge {u, v} belongs to the endpoint with
// the shorter row (ties: the smaller id), and only when that row has at most
// `budget` arcs (any length when budget < 0): the warp's lanes take u's
// neighbours w, binary-search c(v, w) in v's sorted row, and the warp sums
// PR4's minima and ORs PR3's condition.  Work per vertex grows with the
// square of its own (short) row, so hubs cost little.  Edges that pass
// PR1/PR2 in the same call (lo <= 2) are left to k_pr.
constexpr int kPrWarps = 8;

__device__ __forceinline__ int find_in_global(const int2 *row, int len, int x) {
    int lo = 0, hi = len - 1;
    while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int2 e = row[mid];
        if (e.x == x) return e.y;
        if (e.x < x) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

__global__ void __launch_bounds__(kPrWarps * 32)
k_pr34(const DevGraph g, int *par, long long lam, int lo, int level, int budget, int min_len,
       unsigned long long *unions) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    long long local = 0;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < g.n; u += nw) {
        const int u0 = g.rp[u], u1 = g.rp[u + 1], lu = u1 - u0;
        if (lu <= min_len || (budget >= 0 && lu > budget)) continue;
        const long long du = g.deg[u];
        for (int i0 = u0; i0 < u1; i0 += 32) {
            const int i = i0 + lane;
            bool cand = false;
            int v = 0, c = 0;
            if (i < u1) {
                const int2 e = g.adj[i];
                v = e.x;
                c = e.y;
                const int lv = g.rp[v + 1] - g.rp[v];
                cand = lv > lu || (lv == lu && v > u);
                if (cand && lo <= 2) {
                    const long long dv = g.deg[v];
                    const bool pr12 = (lo <= 1 && level >= 1 && (long long)c >= lam) ||
                                      (level >= 2 && 2LL * c > (du < dv ? du : dv));
                    cand = !pr12;
                }
            }
            unsigned todo = __ballot_sync(0xffffffffu, cand);
            while (todo) {
                const int l = __ffs(todo) - 1;
                todo &= todo - 1;
                const int vv = __shfl_sync(0xffffffffu, v, l);
                const long long cc = __shfl_sync(0xffffffffu, c, l);
                const int v0 = g.rp[vv], lv = g.rp[vv + 1] - v0;
                const long long dv = g.deg[vv];
                long long pr4 = 0;
                bool pr3 = false;
                for (int k = u0 + lane; k < u1; k += 32) {
                    const int2 x = g.adj[k];  // w = x.x, c(u, w) = x.y
                    if (x.x == vv) continue;
                    const int cvw = find_in_global(g.adj + v0, lv, x.x);
                    if (cvw == 0) continue;
                    const long long cuw = x.y;
                    if (2 * (cc + cuw) > du && 2 * (cc + cvw) > dv) pr3 = true;
                    pr4 += cuw < cvw ? cuw : cvw;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) pr4 += __shfl_xor_sync(0xffffffffu, pr4, o);
                const bool ok = __any_sync(0xffffffffu, pr3) || (level >= 4 && cc + pr4 >= lam);
                if (ok && lane == 0 && uf_union(par, u, vv)) ++local;
            }
        }
    }
    if (local) atomicAdd(unions, (unsigned long long)local);
}

// PR3/PR4 for rows of at most kPairRow arcs, one warp per vertex u with
// every (owned edge (u, v), neighbour w of u) pair on its own lane: u's row
// and its owned edges go to shared memory, each lane binary-searches w in
// v's row, and PR4's sums and PR3's flags gather per edge in shared memory.
// The same edges and conditions as k_pr34; a short row fills the warp
// instead of one lane per neighbour.
constexpr int kPairRow = 64;

struct Pr34Smem {
    int w[kPairRow];
    int cw[kPairRow];
    int v[kPairRow];
    int cv[kPairRow];
    int v0[kPairRow];
    int lv[kPairRow];
    long long dv[kPairRow];
    unsigned long long pr4[kPairRow];
    int pr3[kPairRow];
};

__global__ void __launch_bounds__(kPrWarps * 32)
k_pr34_pairs(const DevGraph g, int *par, long long lam, int lo, int level, int max_len,
             unsigned long long *unions) {
    __shared__ Pr34Smem smem[kPrWarps];
    Pr34Smem &sm = smem[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    long long local = 0;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < g.n; u += nw) {
        const int u0 = g.rp[u], lu = g.rp[u + 1] - u0;
        if (lu == 0 || lu > max_len) continue;
        const long long du = g.deg[u];
        // u's row, and the edges u owns (the longer row on the other side,
        // ties to the larger id) that PR1/PR2 do not already take
        int ne = 0;
        for (int i0 = 0; i0 < lu; i0 += 32) {
            const int i = i0 + lane;
            bool own = false;
            int v = 0, c = 0, v0 = 0, lv = 0;
            long long dv = 0;
            if (i < lu) {
                const int2 e = g.adj[u0 + i];
                v = e.x;
                c = e.y;
                sm.w[i] = v;
                sm.cw[i] = c;
                v0 = g.rp[v];
                lv = g.rp[v + 1] - v0;
                dv = g.deg[v];
                own = lv > lu || (lv == lu && v > u);
                if (own && lo <= 2)
                    own = !((lo <= 1 && level >= 1 && (long long)c >= lam) ||
                            (level >= 2 && 2LL * c > (du < dv ? du : dv)));
            }
            const unsigned m = __ballot_sync(0xffffffffu, own);
            if (own) {
                const int j = ne + __popc(m & ((1u << lane) - 1u));
                sm.v[j] = v;
                sm.cv[j] = c;
                sm.v0[j] = v0;
                sm.lv[j] = lv;
                sm.dv[j] = dv;
                sm.pr4[j] = 0;
                sm.pr3[j] = 0;
            }
            ne += __popc(m);
        }
        __syncwarp();
        if (ne == 0) continue;
        const int np = ne * lu;
        for (int p = lane; p < np; p += 32) {
            const int j = p / lu, k = p - j * lu;
            const int x = sm.w[k], vv = sm.v[j];
            if (x == vv) continue;
            const int cvw = find_in_global(g.adj + sm.v0[j], sm.lv[j], x);
            if (cvw == 0) continue;
            const long long cuw = sm.cw[k], cc = sm.cv[j];
            if (2 * (cc + cuw) > du && 2 * (cc + cvw) > sm.dv[j]) sm.pr3[j] = 1;
            atomicAdd(&sm.pr4[j], (unsigned long long)(cuw < cvw ? cuw : cvw));
        }
        __syncwarp();
        for (int j = lane; j < ne; j += 32) {
            const bool ok = sm.pr3[j] != 0 || (level >= 4 && (long long)sm.cv[j] + (long long)sm.pr4[j] >= lam);
            if (ok && uf_union(par, u, sm.v[j])) ++local;
        }
        __syncwarp();
    }
    if (local) atomicAdd(unions, (unsigned long long)local);
}

int pr_tests_budget(const DevGraph &g, Work &w, i64 lam, int lo, int level, int budget,
                    cudaStream_t s) {
    if (level <= 0 || lo > level || g.arcs == 0) return MC_OK;
    int blocks = (int)(((g.arcs > g.n ? g.arcs : g.n) + 255) / 256);
    int cap = num_sms() * 16;
    if (blocks > cap) blocks = cap;
    unsigned long long *un = reinterpret_cast<unsigned long long *>(&w.st->unions);
    if (lo <= 2) { ++::mc::g_launches; k_pr<<<blocks, 256, 0, s>>>(g, w.par, lam, lo, level, un); }
    if (level >= 3) {
        long long wb = ((long long)g.n + kPrWarps - 1) / kPrWarps;
        const long long cap = (long long)num_sms() * 8;
        if (wb > cap) wb = cap;
        const int short_len = budget >= 0 && budget < kPairRow ? budget : kPairRow;
        ++::mc::g_launches; k_pr34_pairs<<<(int)wb, kPrWarps * 32, 0, s>>>(g, w.par, lam, lo, level, short_len, un);
        if (budget < 0 || budget > kPairRow) {
            ++::mc::g_launches; k_pr34<<<(int)wb, kPrWarps * 32, 0, s>>>(g, w.par, lam, lo, level, budget, kPairRow, un);
        }
    }
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

}  // namespace mc
