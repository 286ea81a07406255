/*
 * mc.h -- C ABI of libmincut: exact global minimum cut on one GB300 GPU.
 *
 * Method (Henzinger, Noe, Schulz, "Shared-memory Exact Minimum Cuts"):
 *   Alg. 2 (Parallel Minimum Cut): start from an upper bound lambda-hat
 *   (minimum weighted degree, Sec. 2.1/3.1.1, optionally lowered by a
 *   label-propagation clustering bound in the manner of VieCut, Sec. 2.3),
 *   then repeat
 *     - Padberg-Rinaldi local tests against lambda-hat (Sec. 2.2, 2.3),
 *     - many concurrent CAPFOREST scans with priority queues capped at
 *       lambda-hat (Alg. 1, Sec. 3.1.2 Lemma 1, Sec. 3.2), uniting the ends of
 *       every edge whose connectivity certificate reaches lambda-hat,
 *     - a full CAPFOREST scan when nothing was united (Alg. 2, Alg. 3),
 *     - contraction of the united blocks (Sec. 2.1, Sec. 3.2 "Parallel Graph
 *       Contraction"), lowering lambda-hat to the minimum degree,
 *   until one vertex is left.  The smallest cut seen is the minimum cut, and
 *   its side is kept as in Sec. 3.3.
 *
 * All arithmetic on this path is integer and lambda is exact.
 *
 * Graphs are undirected, given as a symmetric CSR with int32 offsets,
 * neighbours and non-negative int32 weights: every edge {u, v} of weight c
 * appears as arc (u -> v, c) in row u and as arc (v -> u, c) in row v.
 * Self-loops and zero weights are dropped, parallel arcs are summed
 * (Sec. 2.1 merges parallel edges the same way).
 *
 * Errors: every call returns MC_OK (0) or a negative MC_E* code; nothing
 * throws across this boundary.  mc_strerror() gives a message, including
 * the CUDA error string for MC_ECUDA.
 *
 * Threads and streams: calls on one mc_graph must not overlap; different
 * graphs may be used from different threads on different streams.
 *
 * Diagnostics: with the environment variable MC_VERBOSE set, mc_min_cut
 * prints one line per round (sizes, unions, lambda-hat, phase times) to
 * stderr; the result does not change.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define MC_OK 0
#define MC_EINVAL (-1)     /* malformed input or arguments (see each call)   */
#define MC_ENOMEM (-2)     /* device or host allocation failed               */
#define MC_ECUDA (-3)      /* a CUDA call failed; mc_strerror has the detail */
#define MC_ETIMEOUT (-4)   /* a bounded device wait gave up                  */
#define MC_EOVERFLOW (-5)  /* a weighted degree or bound does not fit        */
#define MC_EINTERNAL (-6)  /* an internal invariant failed (a bug)           */

/* ---- flags for mc_graph_create ----------------------------------------- */
#define MC_DEVICE_PTRS 1   /* row_ptr/col/w are device pointers              */
#define MC_TRUST_INPUT 2   /* skip the symmetry check (still canonicalised)  */

/* ---- options ------------------------------------------------------------ */
#define MC_PQ_LIFO 0       /* BStack order inside a bucket (Sec. 3.1.3)       */
#define MC_PQ_FIFO 1       /* BQueue order inside a bucket (Sec. 3.1.3)       */

#define MC_BOUND_DEGREE 0  /* lambda-hat = minimum weighted degree            */
#define MC_BOUND_LP 1      /* + label-propagation clustering bound (VieCut)   */
#define MC_BOUND_LEARNED 2 /* + the learned proposer's sweep cut over one level
                              of label-propagation clusters (opt.proposer)   */
#define MC_BOUND_BEST 3    /* + both (the proposer on the LP bound's first
                              level of clusters)                             */

typedef struct mc_options {
    int32_t pq_order;        /* MC_PQ_LIFO (default) or MC_PQ_FIFO             */
    int32_t bound;           /* MC_BOUND_DEGREE (default) or MC_BOUND_LP       */
    int32_t pr_level;        /* Padberg-Rinaldi tests 1..pr_level, 0 = off;
                                PR1/PR2 run every round, PR3/PR4 in rounds whose
                                scans unite < n/4 vertices; default 4           */
    int32_t scans_per_round; /* concurrent CAPFOREST warps, 0 = auto           */
    int32_t region_budget;   /* max vertices touched by one scan, 0 = auto
                                (192; 320 on graphs with >= 48 arcs/vertex;
                                64 on graphs below 2^17 vertices)            */
    int32_t lp_iters;        /* label-propagation sweeps for MC_BOUND_LP, 0=auto*/
    uint64_t seed;           /* start vertices / LP parity                      */
    void *cuda_stream;       /* cudaStream_t to run on; NULL = the graph's own */
    void *proposer;          /* mc_proposer* for MC_BOUND_LEARNED / _BEST      */
    int32_t tail_vertices;   /* once the contracted graph has at most this many
                                vertices and 64 arcs per vertex, its remaining
                                rounds run in one single-warp launch; 0 = the
                                default (256), < 0 = never; at most 4096       */
    int32_t approx_milli;    /* 0 = exact (default).  1..500: Matula's
                                (2+eps)-approximation (Sec. 2.2, 3.1.1): each
                                round unites at lambda-hat = min(best cut,
                                ceil(approx_milli * delta / 1000)), i.e.
                                (1/2 - eps) * delta with eps = 1/2 -
                                approx_milli / 1000; the result is the weight
                                of a real cut, at most 1000 / approx_milli
                                times lambda.  mc_min_cut only: the batched
                                solver always solves exactly                   */
    int32_t visits;          /* concurrent scans: how many scans may scan one
                                vertex (Sec. 3.2 allows a vertex to be visited
                                by several processes); 0 or 1 = once, the
                                first scan owns it and the others blacklist it;
                                k > 1: up to k - 1 more scans scan it, and a
                                scan that scanned a vertex it does not own
                                reports no further alpha cuts; at most 8      */
} mc_options;

/* Per-call statistics (all optional). The ms_* phase times come from CUDA events
 * recorded on the call's stream at the phase boundaries and read once when the call
 * ends (no synchronisation between phases); device idle time between two phases is
 * counted in ms_total only. */
typedef struct mc_stats {
    int32_t rounds;          /* contraction rounds of Alg. 2                    */
    int32_t fallback_rounds; /* rounds that needed the full CAPFOREST scan      */
    int64_t bound_initial;   /* lambda-hat before the first round               */
    int64_t n_input;         /* vertices of the canonical input                 */
    int64_t m_input;         /* undirected edges of the canonical input         */
    double ms_total;         /* device time of the whole call                   */
    double ms_bound;         /* initial bound (degrees / LP / proposer); with
                                the LP bound this includes the exact solve of
                                the clustered remainder, whose phases are also
                                counted below                                  */
    double ms_pr;            /* Padberg-Rinaldi tests                           */
    double ms_capforest;     /* CAPFOREST scans (parallel + fallback)           */
    double ms_contract;      /* union-find flatten, relabel, sort, rebuild      */
    int64_t bytes_alg;       /* algorithmic bytes the method had to move        */
    int64_t scanned_arcs;    /* arcs read by CAPFOREST scans                    */
    int64_t scanned_verts;   /* vertices scanned by CAPFOREST scans             */
    int64_t kernel_launches; /* CUDA kernels launched by the call               */
    int32_t scan_launches;   /* launches of the concurrent-scan kernel          */
    int32_t pad_;
    double ms_scan_kernel;   /* device time of those launches (events)          */
    double ms_tail;          /* single-warp tail solver (see tail_vertices)     */
    int32_t tail_launches;   /* 1 if the tail solver finished the call          */
    int32_t pad2_;
} mc_stats;

typedef struct mc_graph mc_graph; /* opaque; owns its device copies */

/* Fill *opt with the defaults (always succeeds for a non-NULL opt). */
int mc_options_default(mc_options *opt);

/*
 * mc_graph_create -- copy and canonicalise a graph on the current device.
 *   n        vertices, >= 2 (a cut needs two non-empty sides, Sec. 2.1)
 *   row_ptr  n+1 int32 offsets, row_ptr[0] = 0, non-decreasing
 *   col      row_ptr[n] int32 neighbours in [0, n)
 *   w        row_ptr[n] int32 weights >= 0, or NULL for an unweighted graph
 *            (every arc has weight 1; nothing is read or copied for it)
 *   flags    MC_DEVICE_PTRS: the arrays live on the device (read on the
 *            graph's stream); otherwise host memory.  MC_TRUST_INPUT: skip
 *            the symmetry check.
 *   out      receives the new graph; the caller keeps ownership of its arrays
 *            (they are copied) and must call mc_graph_destroy().
 * Errors: MC_EINVAL for n < 2, a bad row_ptr, a neighbour out of range, a
 * negative weight, or (unless trusted) an arc (u,v,c) without its mirror
 * (v,u,c) after merging parallel arcs; MC_EOVERFLOW if parallel arcs sum
 * past INT32_MAX or a weighted degree reaches 2^62; MC_ENOMEM; MC_ECUDA.
 */
int mc_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col,
                    const int32_t *w, int32_t flags, mc_graph **out);

/*
 * mc_graph_destroy -- end a graph.  The device buffers and the stream of the
 * last graph destroyed on a device (one per device, the largest so far) are
 * kept for the next mc_graph_create on that device with at most its vertex
 * and arc counts, which then allocates nothing; they stay held until a larger
 * graph replaces them or the process exits.  Errors: MC_EINVAL for NULL.
 */
int mc_graph_destroy(mc_graph *g);

/* Vertices and undirected edges of the canonical graph. */
int mc_graph_size(const mc_graph *g, int64_t *n, int64_t *m);

/*
 * mc_min_cut -- lambda(G) and one side of a minimum cut (Alg. 2, Sec. 3.3).
 *   opt          NULL for defaults
 *   lambda_out   host int64: the exact minimum cut value
 *   side_bitmap  NULL, or ceil(n/32) uint32 words (host memory, or device
 *                memory if the graph was created with MC_DEVICE_PTRS):
 *                bit v (word v/32, bit v%32) = 1 iff vertex v is on the side
 *                that does not contain vertex 0; unused high bits are 0
 *   stats        NULL or filled
 * A disconnected graph has lambda = 0 and the side is every component but
 * vertex 0's.  The call is synchronous: it returns after the device work.
 * Errors: MC_EINVAL (NULL g/lambda_out), MC_EOVERFLOW (minimum weighted
 * degree >= 2^31 - 3, which the int32 scan arithmetic cannot hold),
 * MC_ECUDA, MC_ETIMEOUT, MC_EINTERNAL.
 */
int mc_min_cut(mc_graph *g, const mc_options *opt, int64_t *lambda_out,
               uint32_t *side_bitmap, mc_stats *stats);

/*
 * mc_batch_min_cut -- lambda for each of G independent graphs.
 *   vtx_off   G+1 int64 vertex offsets (graph g has vtx_off[g+1]-vtx_off[g]
 *             vertices, each >= 2)
 *   arc_off   G+1 int64 arc offsets
 *   row_ptr   concatenated per-graph LOCAL offsets: graph g's n_g+1 entries
 *             start at row_ptr[vtx_off[g] + g] and count from 0
 *   col, w    concatenated per-graph arcs with LOCAL neighbour ids
 *   lambdas   G int64 results (host)
 *   bitmaps   NULL, or per-graph side bitmaps: graph g's ceil(n_g/32) words
 *             start at bitmap_word_off[g] (host)
 *   bitmap_word_off  G+1 int64, required when bitmaps is non-NULL
 * One kernel launch solves the whole batch: one warp per graph, graphs
 * taken largest first (Alg. 2 per graph with full capped scans, PR1/PR2 when
 * opt->pr_level >= 1 and the kernel shape in use runs them, and
 * in-warp contraction).  Self-loops and zero weights are dropped and
 * parallel arcs merged; after that every graph must be symmetric (each arc
 * (u, v, c) has its mirror (v, u, c)), which the kernel checks per graph; a
 * disconnected graph gets lambda 0.  stats: n_input/m_input are totals,
 * ms_total is the kernel's device time.
 * Errors: MC_EINVAL (n_g < 2, bad offsets -- a graph's first offset not 0 or
 * its last not its arc count, refused before any launch, or an offset below
 * its predecessor, found by the kernel before it reads that graph's arcs --,
 * neighbour out of range, negative weight, an arc without its mirror), MC_EOVERFLOW, MC_ENOMEM, MC_ECUDA,
 * MC_EINTERNAL -- the first failing graph's code.
 */
int mc_batch_min_cut(int32_t G, const int64_t *vtx_off, const int64_t *arc_off,
                     const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                     const mc_options *opt, int64_t *lambdas, uint32_t *bitmaps,
                     const int64_t *bitmap_word_off, mc_stats *stats);

/*
 * mc_batch_autotune -- time every batched-kernel shape (warps per block x
 * vertices whose scan state fits in shared memory per warp x whether the
 * in-warp PR1/PR2 tests run, which never changes a lambda) on this batch,
 * keep the fastest for later mc_batch_min_cut calls on the current device
 * of this process, and report it.  Arguments as mc_batch_min_cut;
 * ms_per_shape (max_shapes entries, may be NULL) receives each shape's
 * kernel time.  The shapes' results are not returned.
 */
int mc_batch_autotune(int32_t G, const int64_t *vtx_off, const int64_t *arc_off,
                      const int32_t *row_ptr, const int32_t *col, const int32_t *w,
                      const mc_options *opt, int32_t *best_shape, double *ms_per_shape,
                      int32_t max_shapes);

/*
 * mc_batch_shape_count -- how many batched-kernel shapes mc_batch_autotune
 * chooses from (the valid indices are 0 .. count - 1).  No paper counterpart.
 */
int mc_batch_shape_count(void);

/*
 * mc_batch_set_shape -- choose the batched-kernel shape for later
 * mc_batch_min_cut calls of this process, as mc_batch_autotune does after
 * timing them; -1 returns to the default shape.  Every shape gives the same
 * lambdas; only the time differs.  No paper counterpart.  Returns MC_EINVAL
 * for an index outside -1 .. mc_batch_shape_count() - 1, else MC_OK.
 */
int mc_batch_set_shape(int32_t shape);

/* Message for an error code (thread-local detail for MC_ECUDA). */
const char *mc_strerror(int code);

/*
 * mc_test_fail_alloc_after -- fault-injection hook for tests (no paper
 * counterpart): the device allocation after the next `k` ones fails with
 * MC_ENOMEM, as if the device were full; k < 0 switches the hook off.  The
 * count is process-wide and one-shot (it switches itself off after firing).
 * Returns MC_OK.
 */
int mc_test_fail_alloc_after(int64_t k);

/* ---- learned bound proposer -----------------------------------------------
 * A 3-layer message-passing network (hidden 64, BF16 weights and
 * activations, FP32 sums, tensor-core dense transforms) scores every vertex
 * of a graph; the best sweep cut over the scores is an exact integer cut and
 * therefore an upper bound on lambda.  Its inputs are local degree features
 * and two seeded random vectors smoothed by 32 steps of the lazy random walk
 * (the sides of a sparse cut drift apart).  mc_min_cut runs it on one level
 * of label-propagation clusters of G (MC_BOUND_LEARNED, MC_BOUND_BEST) and
 * uses its cut only if it is below the bound it already has, so lambda never
 * depends on the network.  The paper has no learned component.  Parameters
 * are MC_PROPOSER_PARAMS floats (layout in mc_learn.cu).  Graph arguments are
 * graphs made by mc_graph_create; host arrays unless stated.                */
#define MC_PROPOSER_PARAMS 25409
typedef struct mc_proposer mc_proposer;
/* params: NULL = Glorot-uniform init from `seed` (biases 0). */
int mc_proposer_create(const float *params, uint64_t seed, mc_proposer **out);
int mc_proposer_destroy(mc_proposer *p);
int mc_proposer_get(mc_proposer *p, float *params);
int mc_proposer_set(mc_proposer *p, const float *params);
/* logits (n floats) of the forward pass on g */
int mc_proposer_forward(mc_proposer *p, mc_graph *g, float *logits);
/* polarity-invariant BCE loss of the side bitmap (ceil(n/32) words) and its
 * gradient (MC_PROPOSER_PARAMS floats, may be NULL) */
int mc_proposer_grad(mc_proposer *p, mc_graph *g, const uint32_t *side, double *loss, float *grad);
/* forward + backward + one Adam step (beta 0.9 / 0.999) at learning rate lr */
int mc_proposer_train_step(mc_proposer *p, mc_graph *g, const uint32_t *side, float lr, double *loss);
/* the best sweep cut over the scores: *cut (exact) and its side (bitmap,
 * canonical polarity, may be NULL) */
int mc_proposer_bound(mc_proposer *p, mc_graph *g, int64_t *cut, uint32_t *side);
/* The graph the proposer runs on inside mc_min_cut: `lp_iters` sweeps of
 * label propagation (seed as in mc_step_label_prop) on g, the clusters
 * contracted (Sec. 2.1) with merged weights clamped to g's minimum degree,
 * returned as a new graph *out (caller destroys it); cluster_of (n int32,
 * may be NULL) receives each vertex's cluster.  mc_min_cut uses seed
 * (opt.seed ^ 0x9E37) and lp_iters (opt.lp_iters, 0 = 2).  MC_EINVAL when
 * fewer than two clusters form.                                            */
int mc_graph_coarsen(mc_graph *g, int32_t lp_iters, uint64_t seed, mc_graph **out, int32_t *cluster_of);

/* ---- step-level entry points (same kernels as mc_min_cut) ---------------
 * These expose single steps of the path on a created graph for parity
 * testing.  All arrays are host memory, sized as stated.                  */

/* Canonical CSR of the graph: row_ptr n+1, col/w m2 = 2*m entries, rows
 * sorted by neighbour.  Pass NULL arrays to query nothing but sizes.      */
int mc_graph_export(const mc_graph *g, int32_t *row_ptr, int32_t *col, int32_t *w);

/* Weighted degrees (Sec. 2.1), n int64. */
int mc_step_degrees(mc_graph *g, int64_t *deg);

/* Contract the graph by block labels lab[v] in [0, nc) (Sec. 2.1, every
 * block at once): writes the canonical contracted CSR (row_ptr nc+1,
 * col/w up to 2*m entries, weights clamped to `clamp` if clamp > 0) and
 * its arc count to *arcs_out.                                             */
int mc_step_contract(mc_graph *g, const int32_t *lab, int32_t nc, int64_t clamp,
                     int32_t *row_ptr, int32_t *col, int32_t *w, int64_t *arcs_out);

/* Padberg-Rinaldi tests 1..level against bound `lam` (Sec. 2.2 and 2.3 cite
 * them without stating them).  With d() the weighted degree, edge {u, v}
 * passes
 *   PR1: c(u,v) >= lam;
 *   PR2: 2 c(u,v) > min(d(u), d(v));
 *   PR3: a common neighbour w has 2(c(u,v) + c(u,w)) > d(u) and
 *        2(c(u,v) + c(v,w)) > d(v);
 *   PR4: c(u,v) + sum over common neighbours w of min(c(u,w), c(v,w)) >= lam;
 * and from level 2 on, a vertex whose only two arcs have equal weight joins
 * the smaller of its two neighbours.  PR2 and PR3 are strict because every
 * passing edge is contracted at once.  labels[v] = smallest vertex of v's
 * block in the graph of passing edges. */
int mc_step_pr(mc_graph *g, int64_t lam, int32_t level, int32_t *labels);

/* One round of concurrent capped CAPFOREST scans (Alg. 1) at bound `lam`:
 * labels[v] = smallest vertex of v's union-find block, *lam_out = the bound
 * after the scans' alpha updates, *unions_out = successful unions.         */
int mc_step_capforest(mc_graph *g, int64_t lam, const mc_options *opt,
                      int32_t *labels, int64_t *lam_out, int64_t *unions_out);

/* One round of concurrent capped CAPFOREST scans that scan only the vertices
 * in [lo, hi) -- the rank-local step of the single-graph multi-GPU split:
 * every other vertex counts as blacklisted (Sec. 3.2, Lemma 2 part 3), so
 * it still gathers r-values and can be united, but is never scanned; its row
 * may be empty (a rank holds only its own rows).  Outputs as
 * mc_step_capforest, plus side_bitmap (NULL, or ceil(n/32) words): the
 * vertices of the scan prefix whose alpha lowered the bound (all zero when
 * none did).                                                              */
int mc_step_capforest_range(mc_graph *g, int64_t lam, const mc_options *opt, int32_t lo, int32_t hi,
                            int32_t *labels, int64_t *lam_out, int64_t *unions_out, uint32_t *side_bitmap);

/* One full CAPFOREST scan (Alg. 3) of the whole graph from vertex `start`
 * at bound `lam`, queue capped at lam (Lemma 1): labels[v] = smallest vertex
 * of v's block after uniting every edge whose certificate crosses lam,
 * *lam_out = the bound after the scan's alpha updates, *unions_out = unions.
 * Deterministic for given inputs.                                        */
int mc_step_capforest_full(mc_graph *g, int64_t lam, int32_t start, int32_t *labels,
                           int64_t *lam_out, int64_t *unions_out);

/* `iters` label-propagation sweeps (VieCut's clustering, Sec. 2.3, which
 * does not state the rule).  Labels start as the vertex ids; each sweep has
 * two half-sweeps p = 0, 1, and in half-sweep p every vertex v with
 * parity(seed, sweep, v) = p takes, all at once from the labels as they
 * stood, the label of largest total arc weight among its neighbours (ties to
 * the smaller label; a vertex without neighbours keeps its own), where
 * parity(seed, s, v) = splitmix64(seed ^ splitmix64((s << 32) | v)) & 1.
 * labels: n int32. */
int mc_step_label_prop(mc_graph *g, int32_t iters, uint64_t seed, int32_t *labels);

/* ---- allocation-free full scan -------------------------------------------
 * mc_capforest_full_noalloc -- the full CAPFOREST scan of
 * mc_step_capforest_full without any device allocation, for callers that
 * cannot allocate device memory while running: code that forbids allocation
 * after start-up (a cudaMalloc can synchronise the device or fail on a
 * fragmented heap) or a process whose device memory is held by another
 * allocator.  The paper has no counterpart; it is an interface convenience.
 *   n, arcs    vertices (1..MC_NOALLOC_MAX_N) and arcs (0..MC_NOALLOC_MAX_ARCS)
 *   row_ptr    device int32[n+1] offsets
 *   adj        device int32[2*arcs], 8-byte aligned: (neighbour, weight) per
 *              arc, the layout of mc_graph_export's col/w interleaved; every
 *              edge in both rows, weights >= 1, no self-loops
 *   lam        the bound lambda-hat (> 0) the scan certifies against
 *   start      start vertex in [0, n)
 *   labels     device int32[n] output: smallest vertex of each vertex's block
 *              after the scan's unions
 *   lam_out, unions_out  host, may be NULL: bound after the scan's alpha
 *              updates, and the number of unions
 *   cuda_stream  stream to run on (NULL = default stream); the call returns
 *              after the work has finished
 * All scratch (about 8 MB) is one static device array that each GPU which
 * loads the library keeps until exit.  The first call on a device looks up
 * its address (cudaGetSymbolAddress) -- make that call before any stream
 * capture.  Calls share the array: overlapping calls on one device race and
 * must be serialised by the caller.  Sizes beyond the limits below return
 * MC_EINVAL before any device work.  The arrays are checked on the device
 * before anything they index is touched: bad row offsets (row_ptr[0] != 0,
 * a decrease, row_ptr[n] != arcs), a neighbour outside [0, n), a self-loop or
 * a weight below 1 return MC_EINVAL.  Symmetry is not checked: an
 * asymmetric graph gives meaningless labels, but every access stays inside
 * the arrays.
 */
#define MC_NOALLOC_MAX_N 32768
#define MC_NOALLOC_MAX_ARCS 262144
int mc_capforest_full_noalloc(int32_t n, int64_t arcs, const int32_t *row_ptr, const int32_t *adj,
                              int64_t lam, int32_t start, int32_t *labels, int64_t *lam_out,
                              int64_t *unions_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
