// mc_capforest.cu -- concurrent capped CAPFOREST scans (Alg. 1) and the
// full single scan fallback (Alg. 3).
//
// One warp runs one scan.  Thousands of warps scan at once from seeded start
// vertices; a vertex is scanned by the first scan that claims it in the
// shared owner array T (atomicCAS, the paper's shared visited array with
// "every vertex is visited only once", Sec. 3.2).  A scan that pops a vertex
// owned by another scan blacklists it and moves on without touching it
// (Alg. 1, Lemma 2 part 3).
//
// Per scan, in the warp's shared memory:
//   * a hash table vertex -> r(v) (exact int32 connection weight to the
//     scanned set, saturating) for every vertex the scan touched; the
//     entry holds DONE once the vertex is scanned or blacklisted;
//   * a bucket priority queue over keys min(r, C), C = lambda-hat when the
//     scan starts (Lemma 1, Sec. 3.1.2), with a bitmap of non-empty buckets;
//     bucket lists are LIFO (BStack) or FIFO (BQueue) (Sec. 3.1.3).  Entries
//     are lazy: raising a key pushes a new entry; stale ones are dropped at
//     pop time.  With more keys than buckets the buckets are ranges and a
//     pop walks its bucket for the largest key, so the order stays exact.
// Each arc scan of (x, y, c) with y neither scanned nor blacklisted here:
//   if r(y) < lambda-hat <= r(y) + c: union(x, y)       (Alg. 1)
//   r(y) += c; key(y) = min(r(y), C)  (never lowered)
// Each scanned x updates alpha += c(x) - 2 r(x) = c(S), the cut between the
// scanned set S and the rest, and lowers lambda-hat while S != V (Alg. 1).
// A scan ends when its queue is empty.  Once its table holds `budget`
// vertices it takes no new ones: an arc to a vertex it cannot hold is left
// unscanned -- Lemma 1's argument with that arc's weight lowered to 0, the
// refused vertex never entering the scan -- so the scan goes on over the
// vertices it holds and stops reporting alpha.  Ending a scan early keeps
// every union valid (Lemma 2 part 2).
#include <cstdio>

#include "mc_internal.cuh"
#include "mc_scan.cuh"

namespace mc {

// Start vertices come from a shared cursor over a pseudo-random permutation
// of the vertices (an affine map with a stride coprime to n); each warp takes
// A.grab (<= 32) at a time and scans the ones no scan owns yet.  scan(start, sid, L) runs
// one scan with cap L.
template <class ScanFn>
__device__ void scan_driver(const ScanArgs &A, Counters &cnt, ScanFn scan) {
    const int lane = threadIdx.x & 31;
    const u64 n = (u64)A.g.n;
    while (true) {
        u64 base = 0;
        if (lane == 0) base = atomicAdd(&A.st->cursor, (u64)A.grab);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        u64 idx = base + lane;
        int v = -1;
        bool cand = false;
        if (lane < A.grab && idx < n) {
            v = (int)((A.perm_a * idx + A.perm_b) % n);
            cand = *(volatile int *)&A.T[v] == 0;
        }
        unsigned m = __ballot_sync(0xffffffffu, cand);
        while (m) {
            int l = __ffs(m) - 1;
            m &= m - 1;
            int start = __shfl_sync(0xffffffffu, v, l);
            int t = 0;
            long long L = 0;
            if (lane == 0) {
                t = *(volatile int *)&A.T[start];
                L = ld_volatile_i64(&A.st->lam);
            }
            t = __shfl_sync(0xffffffffu, t, 0);
            L = __shfl_sync(0xffffffffu, L, 0);
            if (t != 0 || L <= 0) continue;
            int sid = 0;
            if (lane == 0) sid = atomicAdd(&A.st->scan_ids, 1) + 1;
            sid = __shfl_sync(0xffffffffu, sid, 0);
            scan(start, sid, L);
        }
    }
    // flush counters: unions are per lane, the rest are warp-uniform
    long long un = cnt.unions;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->unions), (unsigned long long)un);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_arcs), (unsigned long long)cnt.arcs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_verts), (unsigned long long)cnt.verts);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->blacklisted), (unsigned long long)cnt.black);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scans), (unsigned long long)cnt.scans);
    }
}

// Blacklisting at first touch (PRECHECK in scan_one) is off: a vertex another
// scan owns still collects r-value (and can be united by its threshold
// crossing, as in Alg. 1, which blacklists at the pop); measured on RHG 2^20
// and 2^21 the extra unions outweigh the longer scans
constexpr bool kPrecheck = false;

// concurrent scans with the list bucket queue (any cap)
template <int WPB, int HC, int NB, bool MULTI>
__global__ void __launch_bounds__(WPB * 32)
k_capforest(ScanArgs A, int fifo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    ScanSmem<HC, NB> &sm = reinterpret_cast<ScanSmem<HC, NB> *>(smem_raw)[threadIdx.x >> 5];
    HashTable<HC, ScanSmem<HC, NB>> tab{&sm, A.limit};
    SmemQ<HC, NB> q;
    q.head = sm.head;
    q.tail = sm.tail;
    q.bits = sm.bits;
    q.eslot = sm.eslot;
    q.enext = sm.enext;
    q.top = &sm.top;
    q.cap = 2 * HC;
    q.fifo = fifo != 0;
    Counters cnt;
    scan_driver(A, cnt, [&](int start, int sid, long long L) {
        for (int i = lane; i < HC; i += 32) sm.key[i] = -1;
        for (int b = lane; b < NB; b += 32) { sm.head[b] = -1; sm.tail[b] = -1; }
        if (lane < NB / 32) sm.bits[lane] = 0;
        if (lane == 0) { sm.top = 0; sm.used = 0; }
        __syncwarp();
        q.C = (int)(L < (long long)kSat - 1 ? L : (long long)kSat - 1);
        q.coarse = q.C + 1 > NB;
        scan_one<HashTable<HC, ScanSmem<HC, NB>>, SmemQ<HC, NB>, kPrecheck, false, MULTI>(A, tab, q, start, sid, cnt);
    });
}

// concurrent scans with the bitmap bucket queue (cap < NBK at launch; the
// cap only falls during the launch)
template <int WPB, int HC, int NBK, bool MULTI>
__global__ void __launch_bounds__(WPB * 32)
k_capforest_bit(ScanArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    ScanSmemBit<HC, NBK> &sm = reinterpret_cast<ScanSmemBit<HC, NBK> *>(smem_raw)[threadIdx.x >> 5];
    Counters cnt;
    scan_driver(A, cnt, [&](int start, int sid, long long L) {
        for (int i = lane; i < HC; i += 32) sm.key[i] = -1;
        for (int i = lane; i < NBK * (HC / 32); i += 32) sm.bits[i] = 0;
        if (lane == 0) sm.used = 0;
        __syncwarp();
        scan_bit<HC, NBK, MULTI>(A, sm, (int)(L < (long long)NBK - 1 ? L : (long long)NBK - 1), start, sid, cnt);
    });
}

// full scan (Alg. 3): one warp, dense r in global memory, queue pool in
// global memory with one entry per possible push
constexpr int kFullNB = 1024;

__global__ void __launch_bounds__(32)
k_capforest_full(ScanArgs A, int start, int *r, int *eslot, int *enext, int pool_cap, int fifo) {
    __shared__ int head[kFullNB];
    __shared__ int tail[kFullNB];
    __shared__ u32 bits[kFullNB / 32];
    __shared__ int top;
    const int lane = threadIdx.x & 31;
    for (int b = lane; b < kFullNB; b += 32) { head[b] = -1; tail[b] = -1; }
    bits[lane] = 0;
    if (lane == 0) top = 0;
    __syncwarp();
    long long L = ld_volatile_i64(&A.st->lam);
    if (L <= 0) return;
    BucketQ<int, kFullNB> q;
    q.head = head;
    q.tail = tail;
    q.bits = bits;
    q.eslot = eslot;
    q.enext = enext;
    q.top = &top;
    q.cap = pool_cap;
    q.C = (int)(L < (long long)kSat - 1 ? L : (long long)kSat - 1);
    q.coarse = q.C + 1 > kFullNB;
    q.fifo = fifo != 0;
    DenseTable tab{r, 0};
    Counters cnt;
    int sid = 1;
    if (lane == 0) atomicAdd(&A.st->scan_ids, 1);
    scan_one<DenseTable, BucketQ<int, kFullNB>, false, true>(A, tab, q, start, sid, cnt);
    if (lane == 0 && A.pairs) A.st->count = cnt.npairs;
    long long un = cnt.unions;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->unions), (unsigned long long)un);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_arcs), (unsigned long long)cnt.arcs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_verts), (unsigned long long)cnt.verts);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scans), 1ULL);
    }
}

// Full scan of a small graph with a small cap (Alg. 3, n <= 8192, key cap
// C <= 63) on one warp: r, the row offsets, the degrees and one bitmap per key
// over the vertices in shared memory.  A pop takes the smallest vertex of the
// largest key, the oracle's order, so the unions are the oracle's whenever
// lambda-hat does not drop inside the scan.  A queue entry packs into one
// word, (key + 1) << 13 | (8191 - vertex), so the entry to pop is a maximum:
// * once x is popped and before its row is applied, the candidate q (the
//   largest entry left) is searched while x's row is on its way; the row only
//   raises keys, so the next pop is the larger of q and the row's largest
//   move, one warp reduction per 32 arcs and no second search;
// * q's first 32 arcs are loaded one pop ahead and used when q is indeed the
//   next pop (about two pops in three on random and hyperbolic graphs).
// The dependent chain per pop is a few shared-memory loads, one search and
// one reduction per chunk of arcs.
constexpr int kSmallN = 8192;
constexpr int kSmallMaxC = 63;

__host__ __device__ inline size_t small_scan_smem(int n, int C, int kw) {
    return (size_t)(C + 1) * 32 * kw * 4 + 8 * (size_t)n + 4 * (size_t)n + 4 * ((size_t)n + 1);
}

__device__ __forceinline__ unsigned small_entry(int key, int v) {
    return ((unsigned)(key + 1) << 13) | (unsigned)(kSmallN - 1 - v);
}

template <int KW>  // bitmap words per lane and key: 32 * KW words cover the vertices
__global__ void __launch_bounds__(32) k_capforest_small(ScanArgs A, int start, int Cmax) {
    extern __shared__ __align__(16) unsigned char ssm[];
    constexpr unsigned kAll = 0xffffffffu;
    constexpr int Wp = 32 * KW;
    const int lane = threadIdx.x;
    const int n = A.g.n;
    const long long L0 = ld_volatile_i64(&A.st->lam);
    if (lane == 0) atomicAdd(&A.st->scan_ids, 1);
    if (L0 <= 0) return;
    const int C = (int)(L0 < Cmax ? L0 : Cmax);  // Cmax sized the shared memory
    u32 *b0 = reinterpret_cast<u32 *>(ssm);      // (C + 1) x Wp, key-major
    long long *deg = reinterpret_cast<long long *>(b0 + (size_t)(C + 1) * Wp);
    int *r = reinterpret_cast<int *>(deg + n);
    int *rp = r + n;
    for (int i = lane; i < (C + 1) * Wp; i += 32) b0[i] = 0;
    for (int v = lane; v < n; v += 32) { r[v] = 0; rp[v] = A.g.rp[v]; deg[v] = A.g.deg[v]; }
    if (lane == 0) {
        rp[n] = A.g.rp[n];
        b0[start >> 5] = 1u << (start & 31);
    }
    __syncwarp();

    // the largest entry, keys above `top` being empty; lowers top past the
    // keys it finds empty; 0 = none
    int top = 0;
    auto search = [&]() -> unsigned {
        for (; top >= 0; --top) {
            const uint4 *row = reinterpret_cast<const uint4 *>(b0 + (size_t)top * Wp + lane * KW);
            int v = INT_MAX;
#pragma unroll
            for (int j = KW / 4 - 1; j >= 0; --j) {
                const uint4 q = row[j];
                const int base = (lane * KW + 4 * j) * 32 - 1;
                if (q.w) v = base + 96 + __ffs(q.w);
                if (q.z) v = base + 64 + __ffs(q.z);
                if (q.y) v = base + 32 + __ffs(q.y);
                if (q.x) v = base + __ffs(q.x);
            }
            v = (int)__reduce_min_sync(kAll, (unsigned)v);
            if (v != INT_MAX) return small_entry(top, v);
        }
        top = 0;
        return 0u;
    };

    long long L = L0, alpha = 0, best = LLONG_MAX, arcs = 0, npairs = 0;
    int Lj = L <= C ? (int)L : INT_MAX;  // L as the join threshold (no join above C)
    int nS = 0, best_len = 0, unions = 0;
    bool alpha_ok = true;
    unsigned pe = search();
    int spec_v = -1;
    int2 spec_e = make_int2(0, 0);
    while (pe != 0u) {
        if (nS >= n) {  // every vertex popped already: an internal error
            if (lane == 0) atomicOr(&A.st->err, kErrNoProgress);
            break;
        }
        const int p = kSmallN - 1 - (int)(pe & (kSmallN - 1)), Kp = (int)(pe >> 13) - 1;
        const int a0 = rp[p], a1 = rp[p + 1];
        const int rx = r[p];
        const long long dx = deg[p];
        // p's first chunk: loaded one pop ahead, or now
        int2 e = spec_e;
        if (p != spec_v) e = a0 + lane < a1 ? A.g.adj[a0 + lane] : make_int2(0, 0);
        if (lane == 0) {
            b0[(size_t)Kp * Wp + (p >> 5)] &= ~(1u << (p & 31));
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
        arcs += a1 - a0;
        // the candidate before p's row is applied, and its first chunk
        const unsigned qe = search();
        spec_v = kSmallN - 1 - (int)(qe & (kSmallN - 1));
        if (qe != 0u) {
            const int qa0 = rp[spec_v], qa1 = rp[spec_v + 1];
            spec_e = qa0 + lane < qa1 ? A.g.adj[qa0 + lane] : make_int2(0, 0);
        } else {
            spec_v = -1;
        }
        __syncwarp();  // the search reads the bitmaps before p's moves change them
        unsigned be = qe;  // the next pop: the candidate or a larger move
        int xh = p;
        for (int i0 = a0; i0 < a1; i0 += 32) {
            if (i0 != a0) e = i0 + lane < a1 ? A.g.adj[i0 + lane] : make_int2(0, 0);
            const int y = e.x;
            unsigned me = 0u;
            bool join = false;
            if (i0 + lane < a1) {
                const int ro = r[y];
                if (ro != kDone) {
                    const int rn = sat_add(ro, e.y);
                    r[y] = rn;
                    // a certificate min(r, C) only vouches for bounds <= C
                    join = ro < Lj && Lj <= rn;
                    const int ko = ro == 0 ? -1 : (ro < C ? ro : C), kn = rn < C ? rn : C;
                    if (ko != kn) {
                        const u32 bit = 1u << (y & 31);
                        if (ko >= 0) atomicAnd(&b0[(size_t)ko * Wp + (y >> 5)], ~bit);
                        atomicOr(&b0[(size_t)kn * Wp + (y >> 5)], bit);
                        me = small_entry(kn, y);
                    }
                }
            }
            if (A.pairs) {
                const unsigned jm = __ballot_sync(kAll, join);
                if (join) A.pairs[npairs + __popc(jm & ((1u << lane) - 1u))] = ((u64)(u32)p << 32) | (u32)y;
                npairs += __popc(jm);
            } else {
                int rt = INT_MAX;
                if (join && uf_union_root(A.par, xh, y, &rt)) ++unions;
                rt = __reduce_min_sync(kAll, rt);
                if (rt != INT_MAX) xh = rt;
            }
            me = __reduce_max_sync(kAll, me);
            be = me > be ? me : be;
        }
        const int kb = (int)(be >> 13) - 1;
        top = kb > top ? kb : top;
        pe = be;
        __syncwarp();
    }
    if (lane == 0) {
        A.rec_alpha[1] = best;
        A.rec_len[1] = best_len;
        if (A.pairs) A.st->count = npairs;
    }
    unions = (int)__reduce_add_sync(kAll, (unsigned)unions);
    if (lane == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->unions), (unsigned long long)unions);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_arcs), (unsigned long long)arcs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_verts), (unsigned long long)nS);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scans), 1ULL);
    }
}

// ------------------------------------------------ block-wide full scan --
// One thread block runs the whole full scan (Alg. 3 with the Lemma 1 cap).
// The queue keeps, per key 0..C, a bitmap over the vertices (level 0), a
// bitmap over level 0's words (level 1) and one over level 1's words (level
// 2), plus a count per key and a bitmap of the keys that may hold vertices.
// Summary bits are set when a word gains its first vertex and cleared lazily,
// when a pop finds the word below them empty, so they are always a superset.
// A pop takes the smallest vertex of the largest key -- the oracle's order
// (largest key, ties to the smaller vertex) -- so the scan makes the same
// unions as the oracle's whenever lambda-hat does not drop inside it.  The
// popped vertex's row is spread over the block: each arc adds to r(y) (a
// neighbour appears once per row, so r needs no atomics), tests the union
// and moves y to its new key with atomics that only clear level-0 bits and
// only set summary bits, so concurrent moves never lose a vertex.
constexpr int kBlkThreads = 512;

struct BlkArgs {
    int C, W, W1, W2;
    int *r;          // r(v), when not on chip
    u32 *b0, *b1;    // levels 0 and 1, when not on chip
    int on_chip;     // r, levels 0-1, row offsets and degrees in shared memory
    int b1_on_chip;  // otherwise: level 1 in shared memory still (it is small)
};

__host__ __device__ inline size_t blk_smem_bytes(int n, int C, int W, int W1, int W2, bool on_chip,
                                                 bool b1_on_chip = false) {
    size_t b = (size_t)(C + 1) * W2 * 4 + (size_t)(C + 1) * 4 + 32 * 4;  // level 2, counts, key bitmap
    if (!on_chip && b1_on_chip) b += (size_t)(C + 1) * W1 * 4;
    if (on_chip) {
        b += (size_t)(C + 1) * (W + W1) * 4 + 4 * (size_t)n + 4 * ((size_t)n + 1);
        b = (b + 7) / 8 * 8 + 8 * (size_t)n;
    }
    return b;
}

__global__ void __launch_bounds__(kBlkThreads) k_capforest_block(ScanArgs A, int start, BlkArgs B) {
    extern __shared__ __align__(16) unsigned char bsm[];
    __shared__ int s_x, s_a0, s_a1;
    __shared__ long long s_L;
    __shared__ unsigned long long s_np;
    const int n = A.g.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int C = B.C, W = B.W, W1 = B.W1, W2 = B.W2;
    u32 *b2 = reinterpret_cast<u32 *>(bsm);
    int *cnt = reinterpret_cast<int *>(b2 + (size_t)(C + 1) * W2);
    u32 *topb = reinterpret_cast<u32 *>(cnt + C + 1);
    u32 *b0 = B.b0, *b1 = B.b1;
    int *r = B.r;
    const int *rp = A.g.rp;
    const i64 *deg = A.g.deg;
    if (B.on_chip) {
        b0 = topb + 32;
        b1 = b0 + (size_t)(C + 1) * W;
        r = reinterpret_cast<int *>(b1 + (size_t)(C + 1) * W1);
        int *rps = r + n;
        size_t off = (size_t)(reinterpret_cast<unsigned char *>(rps + n + 1) - bsm);
        off = (off + 7) / 8 * 8;
        i64 *degs = reinterpret_cast<i64 *>(bsm + off);
        for (int i = tid; i < (C + 1) * (W + W1); i += kBlkThreads) b0[i] = 0;
        for (int v = tid; v < n; v += kBlkThreads) {
            r[v] = 0;
            rps[v] = A.g.rp[v];
            degs[v] = A.g.deg[v];
        }
        if (tid == 0) rps[n] = A.g.rp[n];
        rp = rps;
        deg = degs;
    } else if (B.b1_on_chip) {
        b1 = topb + 32;
        for (int i = tid; i < (C + 1) * W1; i += kBlkThreads) b1[i] = 0;
    }
    for (int i = tid; i < (C + 1) * W2; i += kBlkThreads) b2[i] = 0;
    for (int i = tid; i <= C; i += kBlkThreads) cnt[i] = 0;
    if (tid < 32) topb[tid] = 0;
    __syncthreads();
    if (tid == 0) {
        // the start vertex, key 0 (r, levels 0-1 off chip arrive zeroed)
        b0[start >> 5] |= 1u << (start & 31);
        b1[start >> 10] |= 1u << ((start >> 5) & 31);
        b2[start >> 15] |= 1u << ((start >> 10) & 31);
        cnt[0] = 1;
        topb[0] = 1u;
        s_np = 0;
        s_L = ld_volatile_i64(&A.st->lam);
        atomicAdd(&A.st->scan_ids, 1);
    }
    __syncthreads();
    if (s_L <= 0) return;
    long long alpha = 0, best = LLONG_MAX, arcs = 0;  // thread 0
    int nS = 0, best_len = 0;
    bool alpha_ok = true;
    while (true) {
        if (wid == 0) {
            // pop: the smallest vertex of the largest key
            int x = -1;
            while (true) {
                const u32 tw = topb[lane];
                const unsigned m = __ballot_sync(0xffffffffu, tw != 0u);
                if (!m) break;
                const int wl = 31 - __clz(m);
                const u32 twv = __shfl_sync(0xffffffffu, tw, wl);
                const int b = wl * 32 + 31 - __clz(twv);
                if (cnt[b] == 0) {
                    __syncwarp();
                    if (lane == 0) topb[b >> 5] &= ~(1u << (b & 31));
                    __syncwarp();
                    continue;
                }
                int found = -1;
                for (int guard = 0; found < 0 && guard <= W1; ++guard) {
                    const u32 w2 = lane < W2 ? b2[(size_t)b * W2 + lane] : 0u;
                    const unsigned m2 = __ballot_sync(0xffffffffu, w2 != 0u);
                    if (!m2) break;
                    const int i2 = __ffs(m2) - 1;
                    const int i1 = i2 * 32 + __ffs(__shfl_sync(0xffffffffu, w2, i2)) - 1;
                    int res = -1;
                    if (lane == 0) {
                        u32 w1 = b1[(size_t)b * W1 + i1];
                        while (w1) {
                            const int i0 = i1 * 32 + __ffs(w1) - 1;
                            const u32 w0 = b0[(size_t)b * W + i0];
                            if (w0) {
                                res = i0 * 32 + __ffs(w0) - 1;
                                b0[(size_t)b * W + i0] = w0 & (w0 - 1u);
                                break;
                            }
                            w1 &= w1 - 1u;  // stale summary bit: that word emptied
                            b1[(size_t)b * W1 + i1] = w1;
                        }
                        if (res < 0) b2[(size_t)b * W2 + i2] &= ~(1u << (i1 & 31));
                        else cnt[b] -= 1;
                    }
                    found = __shfl_sync(0xffffffffu, res, 0);
                    __syncwarp();
                }
                if (found < 0) {  // a count without a vertex: an internal error
                    if (lane == 0) atomicOr(&A.st->err, kErrNoProgress);
                    break;
                }
                x = found;
                break;
            }
            if (lane == 0) {
                if (x >= 0) {
                    const int a0 = rp[x], a1 = rp[x + 1];
                    const long long dx = deg[x];
                    const int rx = r[x];
                    r[x] = kDone;
                    A.T[x] = 1;
                    A.order[x] = nS;
                    ++nS;
                    if (rx >= kSat) alpha_ok = false;
                    alpha += dx - 2LL * rx;
                    if (alpha_ok && nS < n && alpha < s_L) {
                        atomicMin(&A.st->lam, alpha);
                        best = alpha;
                        best_len = nS;
                        s_L = alpha;
                    }
                    s_a0 = a0;
                    s_a1 = a1;
                    arcs += a1 - a0;
                }
                s_x = x;
            }
        }
        __syncthreads();
        const int x = s_x;
        if (x < 0) break;
        const long long L = s_L;
        const int a1 = s_a1;
        for (int i = s_a0 + tid; i < a1; i += kBlkThreads) {
            const int2 e = A.g.adj[i];
            const int y = e.x;
            const int ro = r[y];
            if (ro == kDone) continue;
            const int rn = sat_add(ro, e.y);
            r[y] = rn;
            // a certificate min(r, C) only vouches for bounds <= C
            if ((long long)ro < L && L <= (long long)rn && L <= (long long)C) {
                if (A.pairs) A.pairs[atomicAdd(&s_np, 1ULL)] = ((u64)(u32)x << 32) | (u32)y;
                else if (uf_union(A.par, x, y)) atomicAdd(&s_np, 1ULL);
            }
            const int ko = ro == 0 ? -1 : (ro < C ? ro : C), kn = rn < C ? rn : C;
            if (ko == kn) continue;
            const u32 bit = 1u << (y & 31);
            if (ko >= 0) {
                atomicAnd(&b0[(size_t)ko * W + (y >> 5)], ~bit);
                atomicSub(&cnt[ko], 1);
            }
            if (atomicOr(&b0[(size_t)kn * W + (y >> 5)], bit) == 0u &&
                atomicOr(&b1[(size_t)kn * W1 + (y >> 10)], 1u << ((y >> 5) & 31)) == 0u)
                atomicOr(&b2[(size_t)kn * W2 + (y >> 15)], 1u << ((y >> 10) & 31));
            if (atomicAdd(&cnt[kn], 1) == 0) atomicOr(&topb[kn >> 5], 1u << (kn & 31));
        }
        __syncthreads();
    }
    if (tid == 0) {
        A.rec_alpha[1] = best;
        A.rec_len[1] = best_len;
        if (A.pairs) A.st->count = (long long)s_np;
        else atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->unions), s_np);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_arcs), (unsigned long long)arcs);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scanned_verts), (unsigned long long)nS);
        atomicAdd(reinterpret_cast<unsigned long long *>(&A.st->scans), 1ULL);
    }
}

// launch of the block-wide full scan; `scratch` holds (C + 1) * (W + W1)
// words when the state does not fit on chip, r has n entries (zeroed by the
// caller when off chip)
int launch_full_block(const ScanArgs &A, int start, int C, int *r, u32 *scratch, size_t scratch_words,
                      cudaStream_t s) {
    const int n = A.g.n;
    BlkArgs B;
    B.C = C;
    B.W = (n + 31) / 32;
    B.W1 = (B.W + 31) / 32;
    B.W2 = (B.W1 + 31) / 32;
    const size_t on_chip_bytes = blk_smem_bytes(n, C, B.W, B.W1, B.W2, true);
    B.on_chip = on_chip_bytes <= kBlkOnChipBytes;
    B.b1_on_chip = !B.on_chip && blk_smem_bytes(n, C, B.W, B.W1, B.W2, false, true) <= kBlkOnChipBytes;
    const size_t smem = B.on_chip ? on_chip_bytes : blk_smem_bytes(n, C, B.W, B.W1, B.W2, false, B.b1_on_chip);
    B.r = r;
    B.b0 = scratch;
    B.b1 = scratch + (size_t)(C + 1) * B.W;
    if (!B.on_chip) {
        if ((size_t)(C + 1) * (B.W + B.W1) > scratch_words) return MC_EINTERNAL;
        MC_CUDA(cudaMemsetAsync(scratch, 0, sizeof(u32) * (size_t)(C + 1) * (B.W + B.W1), s));
    }
    static bool attr = false;
    if (!attr) {
        MC_CUDA(cudaFuncSetAttribute(k_capforest_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kBlkOnChipBytes));
        attr = true;
    }
    ++::mc::g_launches; k_capforest_block<<<1, kBlkThreads, smem, s>>>(A, start, B);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

size_t full_block_words(int n, int C) {
    const size_t W = ((size_t)n + 31) / 32, W1 = (W + 31) / 32, W2 = (W1 + 31) / 32;
    if (blk_smem_bytes(n, C, (int)W, (int)W1, (int)W2, true) <= kBlkOnChipBytes) return 0;
    return (size_t)(C + 1) * (W + W1);
}

template <int KW>
static int launch_small_t(const ScanArgs &A, int start, int C, cudaStream_t s) {
    const size_t smem = small_scan_smem(A.g.n, C, KW);
    static bool attr = false;
    if (!attr) {
        MC_CUDA(cudaFuncSetAttribute(k_capforest_small<KW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)small_scan_smem(kSmallN, kSmallMaxC, 8)));
        attr = true;
    }
    ++::mc::g_launches; k_capforest_small<KW><<<1, 32, smem, s>>>(A, start, C);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

static int launch_small(const ScanArgs &A, int start, int C, cudaStream_t s) {
    return A.g.n <= 32 * 32 * 4 ? launch_small_t<4>(A, start, C, s) : launch_small_t<8>(A, start, C, s);
}

// the unions a lone scan recorded (st->count pairs), counted into st->unions
__global__ void k_apply_pairs(const u64 *__restrict__ pairs, Status *st, int *par) {
    const long long np = st->count;
    long long un = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        const u64 p = pairs[i];
        if (uf_union(par, (int)(p >> 32), (int)(p & 0xFFFFFFFFu))) ++un;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) un += __shfl_xor_sync(0xffffffffu, un, o);
    if ((threadIdx.x & 31) == 0 && un)
        atomicAdd(reinterpret_cast<unsigned long long *>(&st->unions), (unsigned long long)un);
}

// smallest scan id whose best alpha equals lambda-hat
// the smallest scan id whose alpha equals the final lambda-hat, and that
// scan's prefix length (read by the last block to finish; its block counter
// `done` comes back to 0)
__global__ void k_best_scan(const i64 *__restrict__ rec_alpha, const int *__restrict__ rec_len, Status *st,
                            unsigned *done) {
    __shared__ bool last;
    const int ns = st->scan_ids;
    const long long lam = st->lam;
    for (int s = 1 + blockIdx.x * blockDim.x + threadIdx.x; s <= ns; s += gridDim.x * blockDim.x)
        if (rec_alpha[s] == lam) atomicMin(&st->best_scan, s);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const int b = *(volatile int *)&st->best_scan;
        st->best_len = b < INT_MAX ? rec_len[b] : 0;
        if (b == INT_MAX) st->best_scan = -1;
        *done = 0;
    }
}

__global__ void k_scan_reset(Status *st) {
    st->cursor = 0;
    st->scan_ids = 0;
    st->best_scan = INT_MAX;
    st->best_len = 0;
}


// Start candidates per cursor grab, and no more warps than grabs: a launch
// lasts as long as its busiest warp, and on graphs of 2^14 vertices and more
// grabs of 16 halve each warp's run of scans (RHG 2^20: the two scan
// launches 0.96 -> 0.88 ms, the solve 1.74 -> 1.68 ms).  Smaller graphs keep 32: more
// warps there mean smaller scan regions and rounds that unite nothing.
static int grab_and_blocks(ScanArgs &A, int blocks, int wpb) {
    A.grab = A.g.n >= 16384 ? 16 : 32;
    int maxb = (A.g.n + A.grab * wpb - 1) / (A.grab * wpb);
    if (maxb < 1) maxb = 1;
    return blocks > maxb ? maxb : blocks;
}

template <int WPB, int HC, int NBK, bool MULTI>
static int launch_parallel_bit_t(const ScanArgs &A, int warps_wanted, cudaStream_t s) {
    const size_t smem = (size_t)WPB * sizeof(ScanSmemBit<HC, NBK>);
    static bool attr_set = false;
    if (!attr_set) {
        MC_CUDA(cudaFuncSetAttribute(k_capforest_bit<WPB, HC, NBK, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr_set = true;
    }
    int per_sm = 0;
    MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_capforest_bit<WPB, HC, NBK, MULTI>, WPB * 32, smem));
    if (per_sm < 1) per_sm = 1;
    int blocks = per_sm * num_sms();
    if (warps_wanted > 0) {
        int b = (warps_wanted + WPB - 1) / WPB;
        if (b < blocks) blocks = b;
    }
    ScanArgs B = A;
    blocks = grab_and_blocks(B, blocks, WPB);
    ++::mc::g_launches; k_capforest_bit<WPB, HC, NBK, MULTI><<<blocks, WPB * 32, smem, s>>>(B);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

template <int WPB, int HC, int NBK>
static int launch_parallel_bit(const ScanArgs &A, int warps_wanted, cudaStream_t s) {
    return A.visits > 1 ? launch_parallel_bit_t<WPB, HC, NBK, true>(A, warps_wanted, s)
                        : launch_parallel_bit_t<WPB, HC, NBK, false>(A, warps_wanted, s);
}

template <int WPB, int HC, int NB, bool MULTI>
static int launch_parallel_t(const ScanArgs &A, int fifo, int warps_wanted, cudaStream_t s) {
    const size_t smem = (size_t)WPB * sizeof(ScanSmem<HC, NB>);
    static bool attr_set = false;
    if (!attr_set) {
        MC_CUDA(cudaFuncSetAttribute(k_capforest<WPB, HC, NB, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
        attr_set = true;
    }
    int per_sm = 0;
    MC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_capforest<WPB, HC, NB, MULTI>, WPB * 32, smem));
    if (per_sm < 1) per_sm = 1;
    int blocks = per_sm * num_sms();
    if (warps_wanted > 0) {
        int b = (warps_wanted + WPB - 1) / WPB;
        if (b < blocks) blocks = b;
    }
    ScanArgs B = A;
    blocks = grab_and_blocks(B, blocks, WPB);
    ++::mc::g_launches; k_capforest<WPB, HC, NB, MULTI><<<blocks, WPB * 32, smem, s>>>(B, fifo);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

template <int WPB, int HC, int NB>
static int launch_parallel(const ScanArgs &A, int fifo, int warps_wanted, cudaStream_t s) {
    return A.visits > 1 ? launch_parallel_t<WPB, HC, NB, true>(A, fifo, warps_wanted, s)
                        : launch_parallel_t<WPB, HC, NB, false>(A, fifo, warps_wanted, s);
}

static u64 gcd_u64(u64 a, u64 b) {
    while (b) { u64 t = a % b; a = b; b = t; }
    return a;
}

static ScanArgs make_args(const DevGraph &g, Work &w, const ScanConfig &cfg) {
    ScanArgs A;
    A.g = g;
    A.par = w.par;
    A.T = w.T;
    A.order = w.order;
    A.st = w.st;
    A.rec_alpha = w.rec_alpha;
    A.rec_len = w.rec_len;
    const u64 n = (u64)(g.n > 0 ? g.n : 1);
    u64 h = (cfg.seed ^ 0x5851F42D4C957F2DULL) + (u64)cfg.round * 0x9E3779B97F4A7C15ULL;
    h ^= h >> 29; h *= 0xBF58476D1CE4E5B9ULL; h ^= h >> 32;
    u64 a = (h % n) | 1;
    while (gcd_u64(a, n) != 1) a = (a + 2) % n == 0 ? 1 : (a + 2) % n;
    if (n == 1) a = 1;
    A.perm_a = a % n == 0 ? 1 : a;
    A.perm_b = (h >> 17) % n;
    A.limit = 0;
    return A;
}

// Hubs (rows longer than kHubArcs) are never scanned by the concurrent
// scans: their owner entry starts at -1, so a pop of a hub fails its claim
// and the hub is passed over, while as a neighbour it is still touched and
// can be united when its r-value crosses lambda-hat.  A scan that passes
// over a vertex is a capped scan of the graph without it, whose connectivities
// are no larger (the unions stay valid), and alpha stays the cut of the
// scanned set S.  One warp would otherwise walk a hub row of 10^5 arcs alone.
constexpr int kHubArcs = 4096;

// owners start at 0 (free) or -1 (never scanned): hubs, and the vertices
// outside [lo, hi) when a rank scans only the vertices it owns (Sec. 3.2:
// a vertex passed over is a blacklisted one, Lemma 2 part 3)
__global__ void k_owner_init(const int *__restrict__ rp, int n, int *T, int *V, int lo, int hi, Status *st) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the scan status (k_scan_reset's fields)
        st->cursor = 0;
        st->scan_ids = 0;
        st->best_scan = INT_MAX;
        st->best_len = 0;
    }
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        T[v] = (rp[v + 1] - rp[v] > kHubArcs || v < lo || v >= hi) ? -1 : 0;
        if (V) V[v] = 0;
    }
}

int capforest_parallel(const DevGraph &g, Work &w, const ScanConfig &cfg, cudaStream_t s) {
    {
        int blocks = (g.n + 255) / 256;
        if (blocks > num_sms() * 16) blocks = num_sms() * 16;
        if (blocks < 1) blocks = 1;
        // extra visits are counted in w.cnt, which no other step of the
        // round uses while the scans run
        const int lo = cfg.lo > 0 ? cfg.lo : 0, hi = cfg.hi >= 0 && cfg.hi < g.n ? cfg.hi : g.n;
        ++::mc::g_launches;
        k_owner_init<<<blocks, 256, 0, s>>>(g.rp, g.n, w.T, cfg.visits > 1 ? w.cnt : nullptr, lo, hi, w.st);
    }
    ScanArgs A = make_args(g, w, cfg);
    A.visits = cfg.visits > 1 ? cfg.visits : 1;
    A.V = w.cnt;
    // default region budget, measured on RHG: 192 touched vertices per scan
    // (one 256-slot table), 320 on graphs averaging >= 48 arcs per vertex;
    // 64 below 2^17 vertices, where the launch lasts as long as its longest
    // scan rather than its total work
    int budget = cfg.budget > 0 ? cfg.budget : (g.n < 131072 ? 64 : (g.arcs >= 48LL * g.n ? 320 : 192));
    constexpr int WPB = 4;
    int rc;
    if (cfg.lam_hint > 0 && cfg.lam_hint < 64 && !cfg.pq_fifo && budget <= 768) {
        // small cap: bitmap queue
        if (budget <= 192) {
            A.limit = budget;
            // as few buckets as the cap needs: less shared memory per warp,
            // more resident warps
            if (cfg.lam_hint < 8) rc = launch_parallel_bit<WPB, 256, 8>(A, cfg.warps, s);
            else if (cfg.lam_hint < 32) rc = launch_parallel_bit<WPB, 256, 32>(A, cfg.warps, s);
            else rc = launch_parallel_bit<WPB, 256, 64>(A, cfg.warps, s);
        } else if (budget <= 384 - 32) {
            A.limit = budget;
            rc = launch_parallel_bit<WPB, 512, 64>(A, cfg.warps, s);
        } else {
            A.limit = budget;
            rc = launch_parallel_bit<WPB, 1024, 64>(A, cfg.warps, s);
        }
    } else if (budget <= 192) {
        A.limit = budget;
        rc = launch_parallel<WPB, 256, 256>(A, cfg.pq_fifo, cfg.warps, s);
    } else if (budget <= 384 - 32) {
        A.limit = budget;
        rc = launch_parallel<WPB, 512, 256>(A, cfg.pq_fifo, cfg.warps, s);
    } else if (budget <= 768) {
        A.limit = budget;
        rc = launch_parallel<WPB, 1024, 256>(A, cfg.pq_fifo, cfg.warps, s);
    } else {
        A.limit = budget < 1536 ? budget : 1536;
        rc = launch_parallel<WPB, 2048, 256>(A, cfg.pq_fifo, cfg.warps, s);
    }
    if (rc != MC_OK) return rc;
    ++::mc::g_launches;
    k_best_scan<<<64, 256, 0, s>>>(w.rec_alpha, w.rec_len, w.st, reinterpret_cast<unsigned *>(w.red + kRedBestDone));
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

// The full-scan kernel for a graph and bound (off the FIFO order): one warp
// with its whole state in shared memory for small graphs under a small cap
// (the short rows leave a block idle, measured faster up to 8192 vertices),
// the block-wide scan while cap and graph are within its limits, else the
// single-warp list-queue scan.  The first two take the largest key, ties to
// the smallest vertex.  Both entry points below pick through here, so the
// allocating and the allocation-free scans run the same kernel.
bool full_scan_is_small(int n, long long cap, bool fifo) {
    return !fifo && cap > 0 && cap <= kSmallMaxC && n <= kSmallN;
}

static int full_scan_dispatch(const ScanArgs &A, int start, long long cap, int fifo, int *r, int *eslot,
                              int *enext, int pool, u32 *blk, size_t blk_words, cudaStream_t s) {
    if (full_scan_is_small(A.g.n, cap, fifo != 0)) return launch_small(A, start, (int)cap, s);
    if (!fifo && cap > 0 && cap <= kBlkMaxCap && A.g.n <= kBlkMaxN)
        return launch_full_block(A, start, (int)cap, r, blk, blk_words, s);
    ++::mc::g_launches; k_capforest_full<<<1, 32, 0, s>>>(A, start, r, eslot, enext, pool, fifo);
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int capforest_full(const DevGraph &g, Work &w, const ScanConfig &cfg, cudaStream_t s) {
    MC_CUDA(cudaMemsetAsync(w.T, 0, sizeof(int) * (size_t)g.n, s));
    MC_CUDA(cudaMemsetAsync(w.fb_r, 0, sizeof(int) * (size_t)g.n, s));
    ++::mc::g_launches; k_scan_reset<<<1, 1, 0, s>>>(w.st);
    ScanArgs A = make_args(g, w, cfg);
    const int start = cfg.start >= 0 && cfg.start < g.n ? cfg.start : (int)(A.perm_b % (u64)(g.n > 0 ? g.n : 1));
    const i64 pool = g.arcs + 2;
    int *eslot = reinterpret_cast<int *>(w.fb_pool);
    int *enext = eslot + pool;
    // the lone scan records its unions (at most one per arc) in the radix
    // key buffer; one parallel pass applies them
    A.pairs = w.keysA;
    MC_CUDA(cudaMemsetAsync(&w.st->count, 0, sizeof(w.st->count), s));
    const long long cap = cfg.lam_hint;
    if (!cfg.pq_fifo && cap > 0 && cap <= kBlkMaxCap && g.n <= kBlkMaxN) {
        const size_t words = full_block_words(g.n, (int)cap);
        if (words > w.blk_words) {
            dev_free(w.blk, s);
            w.blk = nullptr;
            w.blk_words = 0;
            MC_TRY(dev_alloc_n(&w.blk, words, s));
            w.blk_words = words;
        }
    }
    MC_TRY(full_scan_dispatch(A, start, cap, cfg.pq_fifo, w.fb_r, eslot, enext, (int)pool, w.blk, w.blk_words, s));
    {
        int blocks = (int)((g.arcs + 255) / 256);
        if (blocks > num_sms() * 4) blocks = num_sms() * 4;
        if (blocks < 1) blocks = 1;
        ++::mc::g_launches; k_apply_pairs<<<blocks, 256, 0, s>>>(w.keysA, w.st, w.par);
    }
    ++::mc::g_launches;
    k_best_scan<<<1, 32, 0, s>>>(w.rec_alpha, w.rec_len, w.st, reinterpret_cast<unsigned *>(w.red + kRedBestDone));
    MC_CUDA(cudaGetLastError());
    return MC_OK;
}

int capforest_full_raw(const DevGraph &g, int *par, int *T, int *order, Status *st, i64 *rec_alpha,
                       int *rec_len, int *r, int *eslot, int *enext, int pool, u32 *blk, size_t blk_words,
                       int start, cudaStream_t s) {
    ScanArgs A;
    A.g = g;
    A.par = par;
    A.T = T;
    A.order = order;
    A.st = st;
    A.rec_alpha = rec_alpha;
    A.rec_len = rec_len;
    A.perm_a = 1;
    A.perm_b = 0;
    A.limit = 0;
    long long cap = 0;
    MC_CUDA(cudaMemcpyAsync(&cap, &st->lam, sizeof(cap), cudaMemcpyDeviceToHost, s));
    MC_CUDA(cudaStreamSynchronize(s));
    return full_scan_dispatch(A, start, cap, 0, r, eslot, enext, pool, blk, blk_words, s);
}

}  // namespace mc
