// mc_scan.cuh -- one CAPFOREST scan (Alg. 1 / Alg. 3) run by one warp, with
// its bucket priority queue and r-value tables.  Shared by the concurrent
// scan kernel, the full-scan kernels and the per-graph warp solver; the
// design notes are at the top of mc_capforest.cu.
#pragma once

#include "mc_internal.cuh"

namespace mc {

constexpr int kDone = -1;
constexpr int kSat = 0x7FFFFFFE;  // saturation value of r

__device__ __forceinline__ int sat_add(int r, int c) { return r > kSat - c ? kSat : r + c; }

// ------------------------------------------------------- bucket queue ----
template <class Idx, int NB>
struct BucketQ {
    int *head;
    int *tail;
    u32 *bits;
    Idx *eslot;
    Idx *enext;
    int *top;
    int cap;   // pool entries
    int C;     // key cap
    bool coarse;
    bool fifo;
    static constexpr Idx NIL = (Idx)(-1);
    static constexpr int kNBuckets = NB;

    __device__ __forceinline__ int bucket(int k) const {
        return coarse ? (int)(((long long)k * NB) / ((long long)C + 1)) : k;
    }
    __device__ __forceinline__ int nxt(int e) const {
        Idx v = enext[e];
        return v == NIL ? -1 : (int)v;
    }
};

// lanes with `want` push (slot s, key k); all lanes call.  false = no room.
// Lanes pushing into the same bucket are chained in lane order (found with
// match_any), so a push needs no atomics on list heads and the resulting
// order -- hence the scan order among equal keys -- is deterministic.
template <class Idx, int NB>
__device__ bool pq_push(BucketQ<Idx, NB> &q, bool want, int s, int k) {
    const int lane = threadIdx.x & 31;
    unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return true;
    int base = 0;
    if (lane == 0) {
        base = *q.top;
        if (base + __popc(m) > q.cap) base = -1;
        else *q.top = base + __popc(m);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base < 0) return false;
    const int e = base + __popc(m & ((1u << lane) - 1u));
    const int b = want ? q.bucket(k) : -1 - lane;  // distinct dummies for idle lanes
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const unsigned below = peers & ((1u << lane) - 1u);
    const unsigned above = peers & ~((2u << lane) - 1u);
    const int lo_lane = below ? 31 - __clz(below) : lane;  // next lower peer
    const int hi_lane = above ? __ffs(above) - 1 : lane;   // next higher peer
    const int e_lo = __shfl_sync(0xffffffffu, e, lo_lane);
    const int e_hi = __shfl_sync(0xffffffffu, e, hi_lane);
    const bool first = want && !below, last = want && !above;
    int old = -1;
    if (first) old = q.fifo ? q.tail[b] : q.head[b];
    __syncwarp();
    if (want) {
        q.eslot[e] = (Idx)s;
        if (!q.fifo) {
            // LIFO: the highest lane becomes the head, each lane points down
            q.enext[e] = first ? (old < 0 ? q.NIL : (Idx)old) : (Idx)e_lo;
            if (last) q.head[b] = e;
        } else {
            // FIFO: append in lane order after the old tail
            q.enext[e] = last ? q.NIL : (Idx)e_hi;
            if (first) {
                if (old < 0) q.head[b] = e;
                else q.enext[old] = (Idx)e;
            }
            if (last) q.tail[b] = e;
        }
        if (first) atomicOr(&q.bits[b >> 5], 1u << (b & 31));
    }
    __syncwarp();
    return true;
}

// warp-cooperative pop of a maximum key; returns the slot or -1 if empty.
// rv[slot] is the slot's r value or kDone.
template <class Idx, int NB>
__device__ int pq_pop(BucketQ<Idx, NB> &q, const int *rv) {
    const int lane = threadIdx.x & 31;
    while (true) {
        u32 word = lane < NB / 32 ? q.bits[lane] : 0u;
        unsigned m = __ballot_sync(0xffffffffu, word != 0u);
        if (!m) return -1;
        int wl = 31 - __clz(m);
        u32 wv = __shfl_sync(0xffffffffu, word, wl);
        int b = wl * 32 + 31 - __clz(wv);
        int found = -1;
        if (lane == 0) {
            int prev = -1, e = q.head[b];
            int best = -1, bestprev = -1, bestkey = -1;
            while (e >= 0) {
                int s = (int)q.eslot[e];
                int nx = q.nxt(e);
                int r = rv[s];
                int key = r < q.C ? r : q.C;
                bool valid = r != kDone && q.bucket(key) == b;
                if (!valid) {
                    if (prev < 0) q.head[b] = nx; else q.enext[prev] = nx < 0 ? q.NIL : (Idx)nx;
                    if (q.fifo && nx < 0) q.tail[b] = prev;
                    e = nx;
                    continue;
                }
                if (key > bestkey) { bestkey = key; best = e; bestprev = prev; }
                if (!q.coarse || key == q.C) break;
                prev = e;
                e = nx;
            }
            if (best >= 0) {
                int nx = q.nxt(best);
                if (bestprev < 0) q.head[b] = nx; else q.enext[bestprev] = nx < 0 ? q.NIL : (Idx)nx;
                if (q.fifo && nx < 0) q.tail[b] = bestprev;
                found = (int)q.eslot[best];
            }
            if (q.head[b] < 0) {
                q.bits[b >> 5] &= ~(1u << (b & 31));
                q.tail[b] = -1;
            }
        }
        found = __shfl_sync(0xffffffffu, found, 0);
        __syncwarp();
        if (found >= 0) return found;
    }
}

// ------------------------------------------------------------- tables ----
// shared-memory hash table of one warp's scan
template <int HC, int NB>
struct ScanSmem {
    int key[HC];
    int val[HC];
    unsigned short eslot[2 * HC];
    unsigned short enext[2 * HC];
    int head[NB];
    int tail[NB];
    u32 bits[NB / 32];
    int top;
    int used;
};

template <int HC>
struct LogHC;
template <> struct LogHC<256> { static constexpr int v = 8; };
template <> struct LogHC<512> { static constexpr int v = 9; };
template <> struct LogHC<1024> { static constexpr int v = 10; };
template <> struct LogHC<2048> { static constexpr int v = 11; };

template <int HC, class SM>
struct HashTable {
    SM *sm;
    int limit;
    __device__ __forceinline__ int *val() const { return sm->val; }
    // slot of y, inserting it; -1 if the table refuses a new vertex
    __device__ __forceinline__ int find(int y) const {
        volatile int *key = sm->key;
        unsigned h = ((unsigned)y * 2654435761u) >> (32 - LogHC<HC>::v);
        for (int p = 0; p < HC; ++p) {
            int k = key[h];
            if (k == y) return (int)h;
            if (k == -1) {
                if (*(volatile int *)&sm->used >= limit) return -1;
                int old = atomicCAS(&sm->key[h], -1, y);
                if (old == -1) {
                    atomicAdd(&sm->used, 1);
                    sm->val[h] = 0;
                    return (int)h;
                }
                if (old == y) return (int)h;
            }
            h = (h + 1) & (HC - 1);
        }
        return -1;
    }
    __device__ __forceinline__ int vertex(int slot) const { return sm->key[slot]; }
    template <class Q>
    __device__ bool rebuild(Q &q) const;
};

// dense table of a full scan: slot = vertex, r in global or shared memory.
// With `n_rebuild` > 0 a full pool is rebuilt from the n_rebuild vertices
// (every touched, unscanned vertex has r > 0); otherwise the pool must be
// large enough for every push (one per arc).
struct DenseTable {
    int *r;
    int n_rebuild = 0;
    __device__ __forceinline__ int *val() const { return r; }
    __device__ __forceinline__ int find(int y) const { return y; }
    __device__ __forceinline__ int vertex(int slot) const { return slot; }
    template <class Q>
    __device__ bool rebuild(Q &q) const;
};

struct ScanArgs {
    DevGraph g;
    int *par, *T, *order;
    Status *st;
    i64 *rec_alpha;
    int *rec_len;
    u64 perm_a, perm_b;
    int limit;
    // a scan running alone may record its unions (x << 32 | y) here instead
    // of applying them (the scan never reads the union-find, so applying the
    // list afterwards gives the same partition); nullptr = apply at once
    u64 *pairs = nullptr;
    // concurrent scans: scans a vertex may have (1 = its owner only) and the
    // per-vertex count of the extra ones
    int visits = 1;
    int *V = nullptr;
    // start candidates a warp takes from the shared cursor at a time
    int grab = 32;
};

// per-warp totals of one launch (each is at most the graph's arc count, < 2^31)
struct Counters {
    int arcs = 0, verts = 0, unions = 0, black = 0, scans = 0;
    int npairs = 0;  // unions recorded in ScanArgs::pairs
};

// garbage-collect a hash table's queue: rebuild every bucket list from the
// live (touched, not DONE) slots
template <int HC, int NB>
__device__ void pq_rebuild(BucketQ<unsigned short, NB> &q, ScanSmem<HC, NB> &sm) {
    const int lane = threadIdx.x & 31;
    for (int b = lane; b < NB; b += 32) { sm.head[b] = -1; sm.tail[b] = -1; }
    if (lane < NB / 32) sm.bits[lane] = 0;
    if (lane == 0) sm.top = 0;
    __syncwarp();
    for (int i0 = 0; i0 < HC; i0 += 32) {
        int i = i0 + lane;
        int r = sm.val[i];
        bool live = sm.key[i] != -1 && r != kDone;
        pq_push(q, live, i, r < q.C ? r : q.C);
    }
}

// One scan of Alg. 1 from `start` with id `sid` and key cap C.
template <int HC, int NB>
__device__ __forceinline__ bool hash_rebuild(BucketQ<unsigned short, NB> &q, ScanSmem<HC, NB> &sm) {
    pq_rebuild(q, sm);
    return true;
}
template <class Q, class SM>
__device__ __forceinline__ bool hash_rebuild(Q &, SM &) {
    return true;  // the bitmap queue never runs out of room
}
template <int HC, class SM>
template <class Q>
__device__ bool HashTable<HC, SM>::rebuild(Q &q) const {
    return hash_rebuild(q, *sm);
}

template <class Q>
__device__ bool dense_rebuild(const DenseTable &t, Q &q);
template <class Q>
__device__ bool DenseTable::rebuild(Q &q) const {
    return dense_rebuild(*this, q);
}
template <class Q>
__device__ bool dense_rebuild(const DenseTable &t, Q &q) {
    const int lane = threadIdx.x & 31;
    const int n_rebuild = t.n_rebuild;
    const int *r = t.r;
    if (n_rebuild <= 0) return false;
    for (int b = lane; b < Q::kNBuckets; b += 32) { q.head[b] = -1; q.tail[b] = -1; }
    for (int b = lane; b < Q::kNBuckets / 32; b += 32) q.bits[b] = 0;
    if (lane == 0) *q.top = 0;
    __syncwarp();
    for (int v0 = 0; v0 < n_rebuild; v0 += 32) {
        const int v = v0 + lane;
        const int rr = v < n_rebuild ? r[v] : 0;
        const bool live = v < n_rebuild && rr > 0;  // kDone is negative
        if (!pq_push(q, live, v, rr < q.C ? rr : q.C)) return false;
    }
    return true;
}

// ---------------------------------------------------- generic queue ops --
// q_update: lanes with `want` move `slot` from key ko (-1: not queued) to kn.
// q_pop: a slot of maximum key, removed, or -1 when empty.
template <class Idx, int NB>
__device__ __forceinline__ bool q_changed(const BucketQ<Idx, NB> &q, int ko, int kn) {
    return q.bucket(kn) != q.bucket(ko);
}
template <class Idx, int NB>
__device__ __forceinline__ bool q_update(BucketQ<Idx, NB> &q, bool want, int s, int ko, int kn) {
    (void)ko;
    return pq_push(q, want, s, kn);
}
template <class Idx, int NB>
__device__ __forceinline__ int q_pop(BucketQ<Idx, NB> &q, const int *rv) {
    return pq_pop(q, rv);
}

// A scan with PRECHECK looks up the owner of every vertex it touches for the
// first time: a vertex another scan already owns is blacklisted right away
// (Alg. 1's blacklisting, taken before any of its arcs count, so it never
// enters this scan's r-values -- Lemma 2 part 3).
//
// SOLO: the scan runs alone on its graph (a full scan, one warp per graph):
// every claim succeeds, so T is written without an atomic, and lambda-hat
// changes only through this scan, so it is kept in a register.
// MULTI: a vertex another scan owns may still be scanned (A.visits > 1);
// instantiated apart so the common single-visit kernels keep their registers.
template <class Table, class Q, bool PRECHECK = false, bool SOLO = false, bool MULTI = false>
__device__ void scan_one(const ScanArgs &A, Table &tab, Q &q, int start, int sid, Counters &cnt) {
    const int lane = threadIdx.x & 31;
    const int n = A.g.n;
    const int C = q.C;
    int *rv = tab.val();
    {
        int s = lane == 0 ? tab.find(start) : 0;
        s = __shfl_sync(0xffffffffu, s, 0);
        q_update(q, lane == 0, s, -1, 0);
    }
    long long alpha = 0, best = LLONG_MAX;
    // lambda-hat as of the scan's start, lowered by the scan's own alpha: a
    // bound other scans lowered meanwhile is picked up at the next scan (a
    // larger bound is still the weight of a cut, so every union stays valid,
    // and one L2 read per pop is saved)
    long long L_solo = ld_volatile_i64(&A.st->lam);
    int nS = 0, best_len = 0;
    bool alpha_ok = true, stop = false;
    cnt.scans++;
    while (!stop) {
        int s = q_pop(q, rv);
        if (s < 0) break;
        int x = tab.vertex(s);
        int rx = rv[s];
        __syncwarp();
        // the row offsets and degree go out with the claim (wasted on a
        // blacklisted pop, but one round trip instead of two otherwise)
        int old = 0, revisit = 0;
        long long L = 0, dx = 0;
        int a0 = 0, a1 = 0;
        if (lane == 0) {
            rv[s] = kDone;
            a0 = A.g.rp[x];
            a1 = A.g.rp[x + 1];
            dx = A.g.deg[x];
            if (SOLO) {
                A.T[x] = sid;
            } else {
                old = atomicCAS(&A.T[x], 0, sid);
                // another scan owns x: one of its visits > 1 (Sec. 3.2)?
                if (MULTI && old > 0) revisit = atomicAdd(&A.V[x], 1) < A.visits - 1;
            }
        }
        if (!SOLO) {
            old = __shfl_sync(0xffffffffu, old, 0);
            if (MULTI) revisit = __shfl_sync(0xffffffffu, revisit, 0);
            if (old != 0 && !revisit) {
                cnt.black++;
                continue;
            }
            // a vertex this scan does not own is not in its recorded prefix:
            // its later alpha values could not be traced back to a side
            if (MULTI && old != 0) alpha_ok = false;
        }
        if (lane == 0) {
            if (old == 0) A.order[x] = nS;
            L = L_solo;
        }
        L = __shfl_sync(0xffffffffu, L, 0);
        dx = __shfl_sync(0xffffffffu, dx, 0);
        a0 = __shfl_sync(0xffffffffu, a0, 0);
        a1 = __shfl_sync(0xffffffffu, a1, 0);
        ++nS;
        if (rx >= kSat) alpha_ok = false;
        alpha += dx - 2LL * rx;
        if (alpha_ok && nS < n && alpha < L) {
            if (lane == 0) atomicMin(&A.st->lam, alpha);
            if (alpha < best) { best = alpha; best_len = nS; }
            L = alpha;
            L_solo = alpha;
        }
        cnt.verts++;
        cnt.arcs += a1 - a0;
        // unions of this pop all involve x: they start their find from the
        // last root seen for x's set (any member of the set finds its root)
        int xh = x;
        for (int i0 = a0; i0 < a1; i0 += 32) {
            int i = i0 + lane;
            bool v = i < a1;
            int y = 0, c = 0;
            if (v) {
                int2 e = A.g.adj[i];
                y = e.x;
                c = e.y;
            }
            int s2 = v ? tab.find(y) : -1;
            // a full table refuses new vertices: the arc stays unscanned (its
            // weight is 0 in Lemma 1's lowered graph) and alpha is no longer
            // the cut of S, but the scan goes on over the vertices it holds
            if (__any_sync(0xffffffffu, v && s2 < 0)) alpha_ok = false;
            bool push = false, join = false;
            int kn = 0, ko = -1;
            if (s2 >= 0) {
                int r_old = rv[s2];
                if (PRECHECK && r_old == 0 && *(volatile int *)&A.T[y] > 0) {
                    rv[s2] = kDone;  // owned by another scan: blacklisted
                    cnt.black++;
                    r_old = kDone;
                }
                if (r_old != kDone) {
                    int r_new = sat_add(r_old, c);
                    rv[s2] = r_new;
                    // a certificate q = min(r, C) can only vouch for bounds <= C
                    join = (long long)r_old < L && L <= (long long)r_new && L <= (long long)C;
                    const int kold = r_old < C ? r_old : C;
                    kn = r_new < C ? r_new : C;
                    push = r_old == 0 || q_changed(q, kold, kn);
                    ko = r_old == 0 ? -1 : kold;
                }
            }
            if (SOLO && A.pairs) {
                const unsigned jm = __ballot_sync(0xffffffffu, join);
                if (join) A.pairs[cnt.npairs + __popc(jm & ((1u << lane) - 1u))] = ((u64)(u32)x << 32) | (u32)y;
                cnt.npairs += __popc(jm);
            } else {
                int rt = INT_MAX;
                if (join && uf_union_root(A.par, xh, y, &rt)) cnt.unions++;
                rt = __reduce_min_sync(0xffffffffu, rt);
                if (rt != INT_MAX) xh = rt;
            }
            // a full pool is rebuilt from the live slots (they already hold
            // this chunk's new keys); a table that cannot rebuild ends the scan
            if (!q_update(q, push, s2, ko, kn) && !tab.rebuild(q)) {
                stop = true;
                alpha_ok = false;
            }
        }
        __syncwarp();
    }
    if (lane == 0) {
        A.rec_alpha[sid] = best;
        A.rec_len[sid] = best_len;
    }
}

// shared memory of one warp's scan with the bitmap queue: per key, a bitmap
// over the table's slots
template <int HC, int NBK>
struct ScanSmemBit {
    int key[HC];
    int val[HC];
    u32 bits[NBK * (HC / 32)];
    int used;
};

// One capped scan (Alg. 1) of the concurrent rounds with the bitmap queue
// (HC <= 1024 table slots, keys 0..C, C < NBK <= 64): the steps of scan_one
// for a hash table, blacklisting at the pop, with the per-pop chain of
// dependent latencies cut three ways:
// * a queue entry packs into one word, (key + 1) << 10 | (1023 - slot), so the
//   next pop is a maximum: the candidate searched once the popped vertex is
//   removed and before its row is applied, or the row's largest move (keys
//   only rise), one warp reduction per 32 arcs and no search after the row;
// * the candidate's row offsets and owner are loaded one pop ahead: when it
//   is popped its claim and its first 32 arcs leave together;
// * a candidate some other scan owned already when it was looked up is
//   blacklisted at its pop without a claim (ownership never reverts within a
//   round, so the claim would fail); with several visits the claim is kept,
//   it also counts the visits.
// A pop takes a largest key, ties to the lowest slot, as Alg. 1 allows.
template <int HC, int NBK, bool MULTI>
__device__ void scan_bit(const ScanArgs &A, ScanSmemBit<HC, NBK> &sm, int C, int start, int sid, Counters &cnt) {
    static_assert(HC <= 1024 && HC % 32 == 0 && HC / 32 <= 32 && NBK <= 64, "bitmap queue bounds");
    constexpr unsigned kAll = 0xffffffffu;
    constexpr int W = HC / 32;
    const int lane = threadIdx.x & 31;
    HashTable<HC, ScanSmemBit<HC, NBK>> tab{&sm, A.limit};
    int *rv = sm.val;
    u32 *bits = sm.bits;
    {
        int s0 = lane == 0 ? tab.find(start) : 0;
        s0 = __shfl_sync(kAll, s0, 0);
        if (lane == 0) bits[s0 >> 5] |= 1u << (s0 & 31);  // key 0
        __syncwarp();
    }
    int top = 0;  // keys above top are empty
    auto search = [&]() -> unsigned {
        for (; top >= 0; --top) {
            const u32 w = lane < W ? bits[top * W + lane] : 0u;
            const unsigned v = __reduce_min_sync(kAll, w ? (unsigned)(lane * 32 + __ffs(w) - 1) : kAll);
            if (v != kAll) return ((unsigned)(top + 1) << 10) | (1023u - v);
        }
        top = 0;
        return 0u;
    };
    long long alpha = 0;
    // lambda-hat as of the scan's start, lowered by the scan's own alpha (as
    // in scan_one); the scan's best alpha and its prefix go straight to the
    // record (rare)
    long long L = ld_volatile_i64(&A.st->lam);
    int Lj = L <= C ? (int)L : INT_MAX;  // the join threshold: none above C
    if (lane == 0) {
        A.rec_alpha[sid] = LLONG_MAX;
        A.rec_len[sid] = 0;
    }
    int nS = 0;
    bool alpha_ok = true;
    cnt.scans++;
    unsigned pe = search();
    // the candidate's slot (-2 - slot when another scan owned it) and row
    int spec_s = -1, spec_a0 = 0, spec_a1 = 0;
    while (pe != 0u) {
        const int s = 1023 - (int)(pe & 1023u), Kp = (int)(pe >> 10) - 1;
        const int x = tab.vertex(s);
        const int rx = rv[s];
        const bool hit = s == spec_s, owned = s == -2 - spec_s;
        if (lane == 0) {
            bits[Kp * W + (s >> 5)] &= ~(1u << (s & 31));
            rv[s] = kDone;
        }
        int old = 0, revisit = 0, a0 = 0, a1 = 0;
        long long dx = 0;
        int2 e = make_int2(0, 0);
        if (!MULTI && owned) {
            old = 1;  // owned when looked up: blacklisted without a claim
        } else {
            if (hit || owned) {  // owned here: several visits, the claim decides
                a0 = spec_a0;
                a1 = spec_a1;
                if (hit && a0 + lane < a1) e = A.g.adj[a0 + lane];  // with the claim
            } else {
                a0 = A.g.rp[x];
                a1 = A.g.rp[x + 1];
            }
            if (lane == 0) {
                dx = A.g.deg[x];
                old = atomicCAS(&A.T[x], 0, sid);
                // another scan owns x: one of its visits > 1 (Sec. 3.2)?
                if (MULTI && old > 0) revisit = atomicAdd(&A.V[x], 1) < A.visits - 1;
            }
        }
        __syncwarp();  // the pop's bit is cleared before the search
        // the candidate before x's row is applied, its row offsets and owner
        const unsigned qe = search();
        spec_s = 1023 - (int)(qe & 1023u);
        if (qe != 0u) {
            const int vq = tab.vertex(spec_s);
            spec_a0 = A.g.rp[vq];
            spec_a1 = A.g.rp[vq + 1];
            if (*(volatile int *)&A.T[vq] != 0) spec_s = -2 - spec_s;
        } else {
            spec_s = -1;
        }
        old = __shfl_sync(kAll, old, 0);
        if (MULTI) revisit = __shfl_sync(kAll, revisit, 0);
        if (old != 0 && !revisit) {
            cnt.black++;
            pe = qe;
            continue;
        }
        // a vertex this scan does not own is not in its recorded prefix: its
        // later alpha values could not be traced back to a side
        if (MULTI && old != 0) alpha_ok = false;
        if (lane == 0 && old == 0) A.order[x] = nS;
        dx = __shfl_sync(kAll, dx, 0);
        ++nS;
        if (rx >= kSat) alpha_ok = false;
        alpha += dx - 2LL * rx;
        if (alpha_ok && nS < A.g.n && alpha < L) {
            if (lane == 0) {
                atomicMin(&A.st->lam, alpha);
                A.rec_alpha[sid] = alpha;
                A.rec_len[sid] = nS;
            }
            L = alpha;
            Lj = L <= C ? (int)L : INT_MAX;
        }
        cnt.verts++;
        cnt.arcs += a1 - a0;
        unsigned be = qe;  // the next pop: the candidate or a larger move
        int xh = x;        // the last root seen for x's set
        for (int i0 = a0; i0 < a1; i0 += 32) {
            const int i = i0 + lane;
            const bool v = i < a1;
            if (v && (i0 != a0 || !hit)) e = A.g.adj[i];
            const int y = e.x;
            const int s2 = v ? tab.find(y) : -1;
            // a full table refuses new vertices: the arc stays unscanned (its
            // weight is 0 in Lemma 1's lowered graph) and alpha is no longer
            // the cut of S, but the scan goes on over the vertices it holds
            if (__any_sync(kAll, v && s2 < 0)) alpha_ok = false;
            bool join = false;
            unsigned me = 0u;
            if (s2 >= 0) {
                const int ro = rv[s2];
                if (ro != kDone) {
                    const int rn = sat_add(ro, e.y);
                    rv[s2] = rn;
                    // a certificate q = min(r, C) can only vouch for bounds <= C
                    join = ro < Lj && Lj <= rn;
                    const int ko = ro == 0 ? -1 : (ro < C ? ro : C), kn = rn < C ? rn : C;
                    if (ko != kn) {
                        const u32 bit = 1u << (s2 & 31);
                        if (ko >= 0) atomicAnd(&bits[ko * W + (s2 >> 5)], ~bit);
                        atomicOr(&bits[kn * W + (s2 >> 5)], bit);
                        me = ((unsigned)(kn + 1) << 10) | (unsigned)(1023 - s2);
                    }
                }
            }
            int rt = INT_MAX;
            if (join && uf_union_root(A.par, xh, y, &rt)) cnt.unions++;
            rt = __reduce_min_sync(kAll, rt);
            if (rt != INT_MAX) xh = rt;
            me = __reduce_max_sync(kAll, me);
            be = me > be ? me : be;
        }
        const int kb = (int)(be >> 10) - 1;
        top = kb > top ? kb : top;
        pe = be;
        __syncwarp();
    }
}

template <int HC_, int NB_>
struct SmemQ : BucketQ<unsigned short, NB_> {
    static constexpr int kHC = HC_;
    static constexpr int kNB = NB_;
};

}  // namespace mc
