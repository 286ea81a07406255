// graphgen.cpp -- seeded synthetic input graphs.
//
// Inputs only: this file holds none of the minimum-cut method's arithmetic.
// Both the CPU oracle tests and the CUDA path read the graphs it writes.
//
// Families (the paper's workloads and their stand-ins):
//   gg_planted     two G(n,p) blocks joined by a few random cross edges
//   gg_rhg         threshold random hyperbolic graph (Krioukov et al.), the
//                  paper's synthetic family (Appendix A), largest component
//   gg_rmat_kcore  R-MAT graph, symmetrised and deduplicated, reduced to its
//                  k-core and largest component (the paper's k-core practice,
//                  Appendix A), integer weights
//   gg_batch       many small connected weighted graphs of uneven size
//
// All randomness comes from splitmix64 (Steele, Lea, Flood 2014) of a counter,
// so every graph is a pure function of its parameters and seed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <unordered_set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using u64 = uint64_t;
using i64 = int64_t;

inline u64 splitmix64(u64 x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

// uniform double in [0, 1) from a 64-bit hash
inline double u01(u64 h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

// counter-based stream: value k of stream (seed, tag)
inline u64 draw(u64 seed, u64 tag, u64 k) {
    return splitmix64(splitmix64(seed ^ (tag * 0xD1B54A32D192ED03ULL)) + k);
}

struct Graph {
    int n = 0;
    std::vector<int32_t> rp, col, w;
    // batch form (G > 0): per-graph local CSRs concatenated
    int G = 0;
    std::vector<i64> voff, aoff;
};

// Symmetric CSR with sorted rows from undirected edges (u != v, no duplicates).
void build_csr(int n, const std::vector<std::pair<int, int>>& e, const std::vector<int32_t>& ew,
               std::vector<int32_t>& rp, std::vector<int32_t>& col, std::vector<int32_t>& w) {
    std::vector<i64> cnt((size_t)n + 1, 0);
    for (auto& p : e) { cnt[p.first + 1]++; cnt[p.second + 1]++; }
    for (int i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    rp.assign((size_t)n + 1, 0);
    for (int i = 0; i <= n; ++i) rp[i] = (int32_t)cnt[i];
    col.assign((size_t)cnt[n], 0);
    w.assign((size_t)cnt[n], 0);
    std::vector<i64> pos(cnt.begin(), cnt.end() - 1);
    for (size_t k = 0; k < e.size(); ++k) {
        int a = e[k].first, b = e[k].second;
        col[pos[a]] = b; w[pos[a]++] = ew[k];
        col[pos[b]] = a; w[pos[b]++] = ew[k];
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int v = 0; v < n; ++v) {
        i64 lo = rp[v], hi = rp[v + 1];
        std::vector<std::pair<int32_t, int32_t>> row;
        row.reserve((size_t)(hi - lo));
        for (i64 a = lo; a < hi; ++a) row.emplace_back(col[a], w[a]);
        std::sort(row.begin(), row.end());
        for (i64 a = lo; a < hi; ++a) { col[a] = row[a - lo].first; w[a] = row[a - lo].second; }
    }
}

int uf_find(std::vector<int>& p, int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

// Keep the largest connected component; vertices keep their relative order.
void keep_lcc(int& n, std::vector<std::pair<int, int>>& e) {
    std::vector<int> p((size_t)n);
    std::iota(p.begin(), p.end(), 0);
    for (auto& x : e) {
        int a = uf_find(p, x.first), b = uf_find(p, x.second);
        if (a != b) { if (a < b) p[b] = a; else p[a] = b; }
    }
    std::vector<int> sz((size_t)n, 0);
    for (int v = 0; v < n; ++v) sz[uf_find(p, v)]++;
    int best = (int)(std::max_element(sz.begin(), sz.end()) - sz.begin());
    std::vector<int> id((size_t)n, -1);
    int m = 0;
    for (int v = 0; v < n; ++v) if (uf_find(p, v) == best) id[v] = m++;
    std::vector<std::pair<int, int>> out;
    out.reserve(e.size());
    for (auto& x : e)
        if (id[x.first] >= 0) out.emplace_back(id[x.first], id[x.second]);
    e.swap(out);
    n = m;
}

// LSD radix sort of 64-bit keys (11-bit digits over `bits` significant bits).
void radix_sort_u64(std::vector<u64>& a, int bits) {
    std::vector<u64> b(a.size());
    for (int shift = 0; shift < bits; shift += 11) {
        std::vector<size_t> cnt(2049, 0);
        for (u64 x : a) cnt[((x >> shift) & 2047) + 1]++;
        for (int i = 0; i < 2048; ++i) cnt[i + 1] += cnt[i];
        for (u64 x : a) b[cnt[(x >> shift) & 2047]++] = x;
        a.swap(b);
    }
}

// ---------------------------------------------------------------- planted --
Graph* planted(u64 seed, int block_n, double avg_deg, int cross) {
    Graph* g = new Graph;
    int n = 2 * block_n;
    std::vector<std::pair<int, int>> e;
    double p = avg_deg / (double)(block_n - 1);
    u64 ctr = 0;
    for (int blk = 0; blk < 2; ++blk) {
        // geometric skipping over the pairs (v, x), x < v (Batagelj & Brandes 2005)
        const double lq = std::log(1.0 - p);
        long long v = 1, x = -1;
        for (;;) {
            double r = u01(draw(seed, 1 + blk, ctr++));
            x += 1 + (long long)std::floor(std::log(1.0 - r) / lq);
            while (x >= v && v < block_n) { x -= v; ++v; }
            if (v >= block_n) break;
            e.emplace_back(blk * block_n + (int)x, blk * block_n + (int)v);
        }
    }
    std::unordered_set<u64> seen;
    int made = 0;
    while (made < cross) {
        int a = (int)(draw(seed, 3, ctr++) % (u64)block_n);
        int b = block_n + (int)(draw(seed, 3, ctr++) % (u64)block_n);
        u64 key = ((u64)a << 32) | (u64)b;
        if (seen.insert(key).second) { e.emplace_back(a, b); ++made; }
    }
    for (auto& x : e) if (x.first > x.second) std::swap(x.first, x.second);
    std::vector<int32_t> ew(e.size(), 1);
    g->n = n;
    build_csr(n, e, ew, g->rp, g->col, g->w);
    return g;
}

// -------------------------------------------------------------------- rhg --
// Threshold (temperature 0) random hyperbolic graph: n points in a disk of
// radius R, angle uniform, radius with density alpha sinh(alpha r) /
// (cosh(alpha R) - 1), alpha = (gamma - 1) / 2; an edge joins two points at
// hyperbolic distance <= R.  R is set so the expected average degree matches.
struct RHGPoints {
    std::vector<double> r, ch, sh, c, s, th;
};

double dtheta_max(double r1, double r2, double R) {
    if (r1 + r2 <= R) return M_PI;
    double num = std::cosh(r1) * std::cosh(r2) - std::cosh(R);
    double den = std::sinh(r1) * std::sinh(r2);
    double x = num / den;
    if (x <= -1.0) return M_PI;
    if (x >= 1.0) return 0.0;
    return std::acos(x);
}

double radius_quantile(double u, double alpha, double R) {
    return std::acosh(1.0 + u * (std::cosh(alpha * R) - 1.0)) / alpha;
}

// expected average degree for radius R by a quantile-midpoint double integral
double expected_degree(int n, double alpha, double R) {
    const int K = 256;
    std::vector<double> q(K);
    for (int i = 0; i < K; ++i) q[i] = radius_quantile((i + 0.5) / K, alpha, R);
    double acc = 0;
#pragma omp parallel for reduction(+ : acc)
    for (int i = 0; i < K; ++i)
        for (int j = 0; j < K; ++j) acc += dtheta_max(q[i], q[j], R) / M_PI;
    return (double)(n - 1) * acc / ((double)K * K);
}

void rhg_edges(int n, const RHGPoints& P, double R, std::vector<std::pair<int, int>>& e) {
    // radial bands of width 0.5 (the last one ends at R); points sorted by angle
    int nb = std::max(1, (int)std::ceil(R / 0.5));
    std::vector<double> lo(nb + 1);
    for (int b = 0; b <= nb; ++b) lo[b] = std::min(R, 0.5 * b);
    std::vector<std::vector<int>> band(nb);
    for (int i = 0; i < n; ++i) {
        int b = std::min(nb - 1, (int)(P.r[i] / 0.5));
        band[b].push_back(i);
    }
    std::vector<std::vector<double>> bth(nb);
    for (int b = 0; b < nb; ++b) {
        std::sort(band[b].begin(), band[b].end(),
                  [&](int x, int y) { return P.th[x] < P.th[y] || (P.th[x] == P.th[y] && x < y); });
        bth[b].resize(band[b].size());
        for (size_t k = 0; k < band[b].size(); ++k) bth[b][k] = P.th[band[b][k]];
    }
    const double coshR = std::cosh(R);
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    std::vector<std::vector<std::pair<int, int>>> loc((size_t)nt);
#pragma omp parallel
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        auto& out = loc[(size_t)t];
#pragma omp for schedule(dynamic, 4096)
        for (int i = 0; i < n; ++i) {
            for (int b = 0; b < nb; ++b) {
                const auto& ids = band[b];
                if (ids.empty()) continue;
                double d = dtheta_max(P.r[i], lo[b], R) + 1e-9;
                auto scan = [&](double a0, double a1) {
                    size_t k = (size_t)(std::lower_bound(bth[b].begin(), bth[b].end(), a0) - bth[b].begin());
                    for (; k < ids.size() && bth[b][k] <= a1; ++k) {
                        int j = ids[k];
                        if (j <= i) continue;
                        double cosd = P.c[i] * P.c[j] + P.s[i] * P.s[j];
                        double chd = P.ch[i] * P.ch[j] - P.sh[i] * P.sh[j] * cosd;
                        if (chd <= coshR) out.emplace_back(i, j);
                    }
                };
                if (d >= M_PI) {
                    scan(-1.0, 7.0);
                } else {
                    double a0 = P.th[i] - d, a1 = P.th[i] + d;
                    if (a0 < 0) { scan(a0 + 2 * M_PI, 7.0); scan(0.0, a1); }
                    else if (a1 >= 2 * M_PI) { scan(a0, 7.0); scan(0.0, a1 - 2 * M_PI); }
                    else scan(a0, a1);
                }
            }
        }
    }
    e.clear();
    size_t tot = 0;
    for (auto& v : loc) tot += v.size();
    e.reserve(tot);
    for (auto& v : loc) { e.insert(e.end(), v.begin(), v.end()); std::vector<std::pair<int, int>>().swap(v); }
}

void rhg_points(u64 seed, int n, double alpha, double R, RHGPoints& P) {
    P.r.resize(n); P.ch.resize(n); P.sh.resize(n); P.c.resize(n); P.s.resize(n); P.th.resize(n);
#pragma omp parallel for
    for (int i = 0; i < n; ++i) {
        double th = 2 * M_PI * u01(draw(seed, 11, (u64)i));
        double r = radius_quantile(u01(draw(seed, 12, (u64)i)), alpha, R);
        P.th[i] = th; P.r[i] = r;
        P.ch[i] = std::cosh(r); P.sh[i] = std::sinh(r);
        P.c[i] = std::cos(th); P.s[i] = std::sin(th);
    }
}

Graph* rhg(u64 seed, int n, double avg_deg, double gamma) {
    double alpha = (gamma - 1.0) / 2.0;
    // bisection on R for the expected average degree (degree falls with R)
    double lo = 0.5, hi = 2.0 * std::log((double)n) + 20.0;
    for (int it = 0; it < 36; ++it) {
        double mid = 0.5 * (lo + hi);
        if (expected_degree(n, alpha, mid) > avg_deg) lo = mid; else hi = mid;
    }
    double R = 0.5 * (lo + hi);
    RHGPoints P;
    std::vector<std::pair<int, int>> e;
    // one measured correction: k ~ exp(-R/2), so R += 2 ln(measured / target)
    for (int pass = 0; pass < 2; ++pass) {
        rhg_points(seed, n, alpha, R, P);
        rhg_edges(n, P, R, e);
        double meas = 2.0 * (double)e.size() / (double)n;
        if (pass == 0 && meas > 0) {
            if (std::fabs(meas / avg_deg - 1.0) < 0.005) break;
            R += 2.0 * std::log(meas / avg_deg);
        }
    }
    Graph* g = new Graph;
    int m = n;
    keep_lcc(m, e);
    std::vector<int32_t> ew(e.size(), 1);
    g->n = m;
    build_csr(m, e, ew, g->rp, g->col, g->w);
    return g;
}

// ------------------------------------------------------------- rmat kcore --
Graph* rmat_kcore(u64 seed, int scale, int edge_factor, double a, double b, double c, int k,
                  int wmax) {
    const i64 nv = (i64)1 << scale;
    const i64 M = (i64)edge_factor << scale;
    std::vector<u64> keys((size_t)M);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (i64 e = 0; e < M; ++e) {
        u64 u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            double r = u01(draw(seed, 21 + (u64)l, (u64)e));
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | (u64)bu;
            v = (v << 1) | (u64)bv;
        }
        if (u == v) { keys[(size_t)e] = ~0ULL; continue; }
        u64 x = std::min(u, v), y = std::max(u, v);
        keys[(size_t)e] = (x << scale) | y;
    }
    radix_sort_u64(keys, 2 * scale + 1);
    std::vector<std::pair<int, int>> e;
    e.reserve(keys.size());
    u64 last = ~0ULL;
    for (u64 key : keys) {
        if (key == ~0ULL || key == last) continue;
        last = key;
        e.emplace_back((int)(key >> scale), (int)(key & (((u64)1 << scale) - 1)));
    }
    std::vector<u64>().swap(keys);
    // k-core by peeling (unweighted degrees)
    int n = (int)nv;
    std::vector<int32_t> rp, col, w;
    {
        std::vector<int32_t> ones(e.size(), 1);
        build_csr(n, e, ones, rp, col, w);
    }
    std::vector<int> deg((size_t)n), stack;
    std::vector<char> dead((size_t)n, 0);
    for (int v = 0; v < n; ++v) {
        deg[v] = rp[v + 1] - rp[v];
        if (deg[v] < k) { dead[v] = 1; stack.push_back(v); }
    }
    while (!stack.empty()) {
        int v = stack.back();
        stack.pop_back();
        for (i64 q = rp[v]; q < rp[v + 1]; ++q) {
            int x = col[q];
            if (!dead[x] && --deg[x] < k) { dead[x] = 1; stack.push_back(x); }
        }
    }
    std::vector<std::pair<int, int>> kept;
    kept.reserve(e.size());
    for (auto& x : e)
        if (!dead[x.first] && !dead[x.second]) kept.push_back(x);
    std::vector<std::pair<int, int>>().swap(e);
    std::vector<int> id((size_t)n, -1);
    int m = 0;
    for (int v = 0; v < n; ++v) if (!dead[v]) id[v] = m++;
    for (auto& x : kept) { x.first = id[x.first]; x.second = id[x.second]; }
    // map back to original ids for the weight hash after the component step
    std::vector<int> orig((size_t)m);
    for (int v = 0; v < n; ++v) if (id[v] >= 0) orig[id[v]] = v;
    // largest component (keep_lcc relabels in order; remember the mapping)
    std::vector<int> p((size_t)m);
    std::iota(p.begin(), p.end(), 0);
    for (auto& x : kept) {
        int ra = uf_find(p, x.first), rb = uf_find(p, x.second);
        if (ra != rb) { if (ra < rb) p[rb] = ra; else p[ra] = rb; }
    }
    std::vector<int> sz((size_t)m, 0);
    for (int v = 0; v < m; ++v) sz[uf_find(p, v)]++;
    int best = m > 0 ? (int)(std::max_element(sz.begin(), sz.end()) - sz.begin()) : 0;
    std::vector<int> id2((size_t)m, -1);
    int m2 = 0;
    for (int v = 0; v < m; ++v) if (m > 0 && uf_find(p, v) == best) id2[v] = m2++;
    std::vector<std::pair<int, int>> fin;
    std::vector<int32_t> ew;
    fin.reserve(kept.size());
    ew.reserve(kept.size());
    for (auto& x : kept) {
        if (id2[x.first] < 0) continue;
        u64 ou = (u64)orig[x.first], ov = (u64)orig[x.second];
        u64 h = draw(seed, 40, (std::min(ou, ov) << 32) | std::max(ou, ov));
        fin.emplace_back(id2[x.first], id2[x.second]);
        ew.push_back(1 + (int32_t)(h % (u64)wmax));
    }
    Graph* g = new Graph;
    g->n = m2;
    build_csr(m2, fin, ew, g->rp, g->col, g->w);
    return g;
}

// ------------------------------------------------------------------ batch --
// Graph i: n ~ U{nmin..nmax}, average degree d ~ U{dmin..dmax},
// m = max(n - 1, round(n d / 2)) distinct edges: a random spanning tree (each
// vertex of a random order attaches to a uniformly chosen earlier one) plus
// uniform extra pairs; weights U{1..wmax}.
Graph* batch(u64 seed, int G, int nmin, int nmax, int dmin, int dmax, int wmax) {
    Graph* g = new Graph;
    g->G = G;
    std::vector<std::vector<int32_t>> RP((size_t)G), COL((size_t)G), W((size_t)G);
    std::vector<int> N((size_t)G);
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < G; ++i) {
        u64 ctr = 0;
        u64 gs = splitmix64(seed ^ (0xA24BAED4963EE407ULL * (u64)(i + 1)));
        int n = nmin + (int)(draw(gs, 1, ctr++) % (u64)(nmax - nmin + 1));
        int d = dmin + (int)(draw(gs, 1, ctr++) % (u64)(dmax - dmin + 1));
        i64 m = std::max<i64>(n - 1, (i64)std::llround((double)n * d / 2.0));
        m = std::min<i64>(m, (i64)n * (n - 1) / 2);
        std::vector<int> perm((size_t)n);
        std::iota(perm.begin(), perm.end(), 0);
        for (int k = n - 1; k > 0; --k) {
            int j = (int)(draw(gs, 2, ctr++) % (u64)(k + 1));
            std::swap(perm[k], perm[j]);
        }
        std::unordered_set<u64> seen;
        std::vector<std::pair<int, int>> e;
        auto add = [&](int a, int b) {
            if (a == b) return false;
            if (a > b) std::swap(a, b);
            u64 key = ((u64)a << 32) | (u64)b;
            if (!seen.insert(key).second) return false;
            e.emplace_back(a, b);
            return true;
        };
        for (int k = 1; k < n; ++k) {
            int j = (int)(draw(gs, 3, ctr++) % (u64)k);
            add(perm[k], perm[j]);
        }
        while ((i64)e.size() < m) {
            int a = (int)(draw(gs, 4, ctr++) % (u64)n);
            int b = (int)(draw(gs, 4, ctr++) % (u64)n);
            add(a, b);
        }
        std::sort(e.begin(), e.end());
        std::vector<int32_t> ew(e.size());
        for (size_t k = 0; k < e.size(); ++k) ew[k] = 1 + (int32_t)(draw(gs, 5, k) % (u64)wmax);
        build_csr(n, e, ew, RP[i], COL[i], W[i]);
        N[i] = n;
    }
    g->voff.assign((size_t)G + 1, 0);
    g->aoff.assign((size_t)G + 1, 0);
    for (int i = 0; i < G; ++i) {
        g->voff[i + 1] = g->voff[i] + N[i];
        g->aoff[i + 1] = g->aoff[i] + (i64)COL[i].size();
    }
    g->n = (int)g->voff[G];
    g->rp.reserve((size_t)g->n + G);
    for (int i = 0; i < G; ++i) {
        g->rp.insert(g->rp.end(), RP[i].begin(), RP[i].end());
        g->col.insert(g->col.end(), COL[i].begin(), COL[i].end());
        g->w.insert(g->w.end(), W[i].begin(), W[i].end());
    }
    return g;
}

}  // namespace

extern "C" {

void* gg_planted(u64 seed, int block_n, double avg_deg, int cross) {
    return planted(seed, block_n, avg_deg, cross);
}
void* gg_rhg(u64 seed, int n, double avg_deg, double gamma) { return rhg(seed, n, avg_deg, gamma); }
void* gg_rmat_kcore(u64 seed, int scale, int edge_factor, double a, double b, double c, int k,
                    int wmax) {
    return rmat_kcore(seed, scale, edge_factor, a, b, c, k, wmax);
}
void* gg_batch(u64 seed, int G, int nmin, int nmax, int dmin, int dmax, int wmax) {
    return batch(seed, G, nmin, nmax, dmin, dmax, wmax);
}
int gg_n(void* h) { return ((Graph*)h)->n; }
long long gg_rp_len(void* h) { return (long long)((Graph*)h)->rp.size(); }
long long gg_arcs(void* h) { return (long long)((Graph*)h)->col.size(); }
int gg_graphs(void* h) { return ((Graph*)h)->G; }
void gg_copy(void* h, int32_t* rp, int32_t* col, int32_t* w, int64_t* voff, int64_t* aoff) {
    Graph* g = (Graph*)h;
    std::memcpy(rp, g->rp.data(), g->rp.size() * sizeof(int32_t));
    if (!g->col.empty()) {
        std::memcpy(col, g->col.data(), g->col.size() * sizeof(int32_t));
        std::memcpy(w, g->w.data(), g->w.size() * sizeof(int32_t));
    }
    if (g->G > 0 && voff && aoff) {
        std::memcpy(voff, g->voff.data(), g->voff.size() * sizeof(int64_t));
        std::memcpy(aoff, g->aoff.data(), g->aoff.size() * sizeof(int64_t));
    }
}
void gg_free(void* h) { delete (Graph*)h; }
}
