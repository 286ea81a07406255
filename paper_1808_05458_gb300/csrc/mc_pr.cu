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
// One thread per arc (u < v).  PR3/PR4 walk the shorter of the two sorted
// rows and binary-search each neighbour in the longer one, only when the
// shorter row has at most `budget` arcs (all rows when budget < 0).
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

__global__ void k_pr(const DevGraph g, int *par, long long lam, int lo, int level, int budget,
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
        if (!ok && level >= 3) {
            const int lu = g.rp[u + 1] - g.rp[u], lv = g.rp[v + 1] - g.rp[v];
            const int a = lu <= lv ? u : v, b = lu <= lv ? v : u;
            const int la = lu <= lv ? lu : lv;
            if (budget < 0 || la <= budget) {
                long long pr4 = c;
                for (int k = g.rp[a]; k < g.rp[a + 1] && !ok; ++k) {
                    const int2 x = g.adj[k];
                    if (x.x == b) continue;
                    const int cb = row_weight(g.rp, g.adj, b, x.x);
                    if (cb == 0) continue;
                    // weights to the common neighbour from u and from v
                    const long long cuw = (a == u) ? x.y : cb;
                    const long long cvw = (a == u) ? cb : x.y;
                    if (2 * (c + cuw) > du && 2 * (c + cvw) > dv) ok = true;
                    pr4 += cuw < cvw ? cuw : cvw;
                    if (level >= 4 && pr4 >= lam) ok = true;  // early exit
                }
                if (!ok && level >= 4 && pr4 >= lam) ok = true;
            }
        }
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

int pr_tests_budget(const DevGraph &g, Work &w, i64 lam, int lo, int level, int budget,
                    cudaStream_t s) {
    if (level <= 0 || lo > level || g.arcs == 0) return MC_OK;
    int blocks = (int)(((g.arcs > g.n ? g.arcs : g.n) + 255) / 256);
    int cap = num_sms() * 16;
    if (blocks > cap) blocks = cap;
    ++::mc::g_launches; k_pr<<<blocks, 256, 0, s>>>(g, w.par, lam, lo, level, budget,
                                reinterpret_cast<unsigned long long *>(&w.st->unions));
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int pr_tests(const DevGraph &g, Work &w, i64 lam, int level, cudaStream_t s) {
    return pr_tests_budget(g, w, lam, 1, level, 64, s);
}

}  // namespace mc
