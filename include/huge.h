/*
 * huge.h — C ABI of a single-GPU (B300, sm_103a) subgraph enumerator following HUGE
 * (Yang et al., "HUGE: An Efficient and Scalable Subgraph Enumeration System", SIGMOD 2021).
 *
 * The hot path is the paper's PULL-EXTEND operator (Sec. 4.2 and Alg. 4: extend each partial
 * match by the intersection of its bound vertices' sorted adjacency lists, Sec. 3.1 Eq. 2),
 * with the symmetry-breaking filter (Sec. 2) fused in, plus PUSH-JOIN (Sec. 4.2-4.3: a hash
 * join of two partial-match sets on their shared query vertices), run under the
 * DFS/BFS-adaptive bounded-memory scheduler (Sec. 5.2, Alg. 5) with work stealing
 * (Sec. 5.3). Counts are exact int64.
 *
 * Conventions for every function below:
 *  - Return value: HUGE_OK (0) or one of the HUGE_E* codes; huge_last_error() then returns a
 *    thread-local, human-readable message. Output arguments are written only on success.
 *  - Pointers marked "host" must be host memory; "device" must be device memory of the current
 *    CUDA device. The library never takes ownership of caller buffers; it copies what it keeps.
 *  - Objects (huge_graph_t, huge_plan_t, huge_mlp_t) are opaque and owned by the library until
 *    the matching *_free call. A plan must not outlive its graph.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream). Calls return
 *    after the result has been copied back (they synchronise the stream).
 *  - Not thread-safe on one object. A graph and every plan made on it count as one object here:
 *    they share the graph's device workspace, so calls that use the same graph (planning with
 *    the sampling estimator, enumeration, autotuning, root features, hub-bitmap and residency
 *    changes) must not overlap. Different graphs may be used from different threads.
 */
#ifndef HUGE_H
#define HUGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define HUGE_OK 0
#define HUGE_EINVAL 1    /* malformed graph/query/order/partial order, bad argument */
#define HUGE_ENOMEM 2    /* mem_bound below the plan's minimum, or device allocation failed */
#define HUGE_EOVERFLOW 3 /* an exact count would not fit in int64 */
#define HUGE_ETIMEOUT 4  /* a bounded device wait gave up */
#define HUGE_ECUDA 5     /* a CUDA runtime call failed */
#define HUGE_ERANGE 6    /* LIST output larger than the sink and no drain callback */

#define HUGE_MAX_QUERY_VERTICES 8

/* ---- huge_graph_load flags ---- */
#define HUGE_RELABEL_BY_DEGREE 1u /* relabel ids by (degree, id) ascending (Sec. 2) */
#define HUGE_TRUST_SORTED 2u      /* skip validation of the CSR (caller guarantees it) */
#define HUGE_DIRECTED 4u          /* adj holds out-lists of a directed graph; queries take arcs */

/* ---- huge_plan flags ---- */
#define HUGE_PLAN_PLAIN 0u       /* Alg. 1 with the sampling cardinality estimator */
#define HUGE_PLAN_LEARNED 1u     /* Alg. 1 with the learned MLP estimator (needs a model) */
#define HUGE_PLAN_EXTEND_ONLY 2u /* only complete star joins (PULL-EXTEND chains) */
#define HUGE_PLAN_TREE_VERIFY 4u /* spanning-tree EXTENDs + verify-only EXTENDs (Sec. 5.2) */
#define HUGE_PLAN_FORCE_JOIN 8u  /* best plan whose top operator is a PUSH-JOIN */
#define HUGE_PLAN_DIRECTED 16u   /* huge_plan_offline only: the query edges are arcs (plans on a
                                    graph take this from the graph's HUGE_DIRECTED) */

/* ---- enumeration modes ---- */
#define HUGE_COUNT 0
#define HUGE_LIST 1

/* ---- huge_enum_opts_t.flags ---- */
#define HUGE_EF_STATS 1u    /* also count algorithmic list bytes (slower; for measurement) */
#define HUGE_EF_NO_STEAL 2u /* disable work stealing between warps */

typedef struct huge_graph huge_graph_t;
typedef struct huge_plan huge_plan_t;
typedef struct huge_mlp huge_mlp_t;

/*
 * LIST sink. `rows` is device memory for capacity_rows rows of k uint32 (row-major); column v
 * of a row holds f(v), the data vertex matched to query vertex v (query-vertex order, not
 * matching order). Row order is unspecified. When the buffer is full the library calls
 * drain(ctx, rows, nrows) (rows[0..nrows) are complete matches, device memory, valid only
 * during the call) and then reuses the buffer; at the end it drains the remainder. With
 * drain == NULL, more matches than capacity_rows fail with HUGE_ERANGE.
 */
typedef void (*huge_drain_fn)(void *ctx, const uint32_t *rows, uint64_t nrows);
typedef struct {
    uint32_t *rows;
    uint64_t capacity_rows;
    huge_drain_fn drain;
    void *ctx;
} huge_sink_t;

/* Measurements of one huge_enumerate_ex call. */
typedef struct {
    int64_t level_rows[16];  /* partial matches per level: [0] roots, [i] rows after operator i */
    int32_t nlevels;         /* number of valid entries in level_rows */
    uint64_t intersections;  /* EXTEND applications (one per input partial match) */
    uint64_t list_bytes;     /* algorithmic bytes (HUGE_EF_STATS only; else 0) */
    uint64_t peak_bytes;     /* device bytes held for intermediate results */
    double device_ms;        /* device time of the enumeration kernels (CUDA events) */
    uint32_t level_cap;      /* rows per level per warp used */
    uint32_t warps;          /* resident warps of the persistent kernel */
    uint32_t launches;       /* kernels launched */
} huge_stats_t;

/* Options of huge_enumerate_ex; zero-initialise for defaults. */
typedef struct {
    uint32_t root_begin;  /* restrict f(v_0) to [root_begin, root_end); root_end 0 = all */
    uint32_t root_end;
    const uint32_t *roots; /* host; if non-NULL, enumerate exactly these roots instead */
    uint64_t nroots;
    uint32_t flags;        /* HUGE_EF_* */
    uint32_t level_cap;    /* rows per level per warp (multiple of 32); 0 = from mem_bound */
    uint32_t chunk_roots;  /* target roots per root task; 0 = degree-balanced automatic */
    const float *root_weights; /* host, n entries: work estimate per root for chunking, or NULL */
    uint32_t time_limit_ms; /* device time limit per launch (0 = 600 s); beyond it HUGE_ETIMEOUT */
    uint32_t variant;      /* intersection of the last operator: 0 tuned/default, 1 binary search
                              only, r >= 2 merge path when the two shortest lists differ <= r x */
    int64_t *per_root;     /* reserved, must be NULL */
} huge_enum_opts_t;

/* ======================================================================================= */
/* Graph                                                                                   */
/* ======================================================================================= */

/*
 * Loads an unlabelled undirected data graph given as CSR (Sec. 2 "Graph Notations"; Sec. 7
 * keeps graphs in CSR): offsets[n+1] (host, uint64, offsets[0] = 0, offsets[n] = nnz) and
 * adj[nnz] (host, uint32). Every list must be strictly increasing, contain no self-loop and
 * only ids < n, and the graph must be symmetric (u in N(v) iff v in N(u)); with
 * HUGE_TRUST_SORTED these checks are skipped. nnz and n must be < 2^32 - 1. With
 * HUGE_RELABEL_BY_DEGREE the library renames vertices so that a smaller degree gets a smaller
 * id, ties by the original id (the total order of Sec. 2 used by symmetry breaking); counts
 * are then in the new ids. The CSR is copied to the device; the caller keeps its buffers.
 * With HUGE_DIRECTED the graph is directed (Sec. 2: direction carries over to the method):
 * adj[offsets[v]..offsets[v+1]) are the heads of the arcs leaving v (no symmetry required,
 * 2 nnz < 2^32 - 1); the library also keeps every in-list, relabels by in + out degree, and
 * every plan on the graph reads its query edges (a, b) as arcs a -> b, each of which a match
 * must map to an arc.
 * Errors: HUGE_EINVAL (malformed input), HUGE_ENOMEM / HUGE_ECUDA (device).
 */
int huge_graph_load(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz,
                    uint32_t flags, huge_graph_t **out);
/*
 * Labelled data graph (Sec. 2: the method carries over to labelled graphs; a match must also
 * map each labelled query vertex to a data vertex of the same label). labels (host, n entries,
 * each < nlabels, original ids) is copied. The library renumbers the vertices by (label,
 * degree, id) with HUGE_RELABEL_BY_DEGREE, else by (label, id), so that every label owns one
 * contiguous id range; a labelled query vertex is then an id-range bound on its EXTEND step
 * (and on the roots) next to the partial-order bounds. huge_graph_new_ids reports the ids.
 * Errors: as huge_graph_load; HUGE_EINVAL for a label >= nlabels or nlabels outside 1..2^24.
 */
int huge_graph_load_labeled(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t nnz,
                            const uint32_t *labels, uint32_t nlabels, uint32_t flags, huge_graph_t **out);
/* nlabels (0 for an unlabelled graph) and, if lstart is not NULL (host, nlabels + 1 entries),
 * the id ranges: label L owns the new ids [lstart[L], lstart[L + 1]). */
int huge_graph_label_ranges(const huge_graph_t *g, uint32_t *nlabels, uint32_t *lstart);
int huge_graph_free(huge_graph_t *g);
/* n, nnz (= 2|E|) and maximum degree D_G of a loaded graph (host outputs; NULL to skip). */
int huge_graph_info(const huge_graph_t *g, uint32_t *n, uint64_t *nnz, uint32_t *max_degree);
/* new_of_old[n] (host): the relabelling applied at load (identity without the flag). */
int huge_graph_new_ids(const huge_graph_t *g, uint32_t *new_of_old);
/*
 * Degree-bucket intersection support (Sec. 3.1 Eq. 2 leaves the intersection method open):
 * the library keeps an n-bit adjacency bitmap on the device for each high-degree vertex ("hub")
 * and tests a candidate against a hub's list with one bit probe instead of a search; lists of
 * the other vertices are searched or merged. This (re)builds the bitmaps of every vertex of
 * degree >= min_degree, highest degree first, while their total stays within max_bytes
 * (device memory held by the graph until it is freed or rebuilt). min_degree 0 or max_bytes
 * below one row (n/8 bytes) removes them; min_degree UINT32_MAX selects the default threshold
 * max(256, n/1024). huge_graph_load builds them with that default and max_bytes = 4 GiB.
 * Counts never depend on this setting, only the speed. Errors: HUGE_ENOMEM, HUGE_ECUDA.
 */
int huge_graph_set_hub_bitmaps(huge_graph_t *g, uint32_t min_degree, uint64_t max_bytes);
/*
 * Out-of-core adjacency (Sec. 4.4 keeps a graph larger than one machine's memory remote and
 * caches adjacency lists locally; here the remote side is host memory and the cache is HBM):
 * moves the graph's adjacency array into managed memory, keeps at most its last hbm_bytes (whole
 * 2 MiB pages, or the whole array when the budget covers it: under degree ordering the lists of
 * the highest-degree vertices, the ones intersections read most) preferred in HBM and
 * prefetched there, and leaves the rest preferred in host memory
 * and mapped for the device, which the same kernels then read across the host link. Offsets,
 * hub bitmaps and intermediate results stay in HBM. May be called again to change the budget;
 * UINT64_MAX keeps the whole array in HBM. *resident_bytes (host, may be NULL) receives the
 * adjacency bytes placed in HBM. The managed array does not come from the allocator hook.
 * Counts never depend on the placement, only the speed. Errors: HUGE_ENOMEM, HUGE_ECUDA.
 */
int huge_graph_set_residency(huge_graph_t *g, uint64_t hbm_bytes, uint64_t *resident_bytes);
/* Number of hub bitmaps, the degree threshold used and the device bytes they hold (host). */
int huge_graph_hub_info(const huge_graph_t *g, uint32_t *count, uint32_t *min_degree, uint64_t *bytes);

/* ======================================================================================= */
/* Plan                                                                                    */
/* ======================================================================================= */

/*
 * Builds an execution plan for the query graph q = (nq vertices, mq edges given as 2*mq
 * vertex ids in q_edges, host). The query must be connected, simple, with nq <= 8.
 *  - order (host, nq entries) or NULL: with an order the plan is the EXTEND chain matching
 *    order[0], order[1], ... (each prefix must be connected; Sec. 3.1, Eq. 2); with NULL the
 *    optimiser of Alg. 1 picks the join order and Eq. 3 picks EXTEND or PUSH-JOIN for each
 *    join.
 *  - po_pairs (host, 2*npo entries, pairs (a, b) meaning f(a) < f(b)) with npo >= 0, or
 *    npo = -1 for the automatic symmetry-breaking partial order (Sec. 2): one match per
 *    automorphism class of q.
 *  - flags: HUGE_PLAN_*.
 * Cardinality estimates for the optimiser run on the GPU (sampling) unless the flags select
 * the learned estimator; huge_plan_ex takes the model.
 * Errors: HUGE_EINVAL (disconnected/oversized query, bad order, partial order not a DAG).
 */
int huge_plan(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
              const uint32_t *order, const uint32_t *po_pairs, int32_t npo, uint32_t flags,
              huge_plan_t **out);
int huge_plan_ex(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
                 const uint32_t *order, const uint32_t *po_pairs, int32_t npo, uint32_t flags,
                 const huge_mlp_t *model, huge_plan_t **out);
/*
 * As huge_plan_ex for a labelled query: q_labels (host, nq entries) gives each query vertex's
 * label, or HUGE_ANY_LABEL for a vertex any data vertex may match; NULL = unlabelled. The
 * automatic partial order (npo = -1) then breaks only the label-preserving automorphisms.
 * The graph must have been loaded with labels (else HUGE_EINVAL).
 */
#define HUGE_ANY_LABEL 0xffffffffu
int huge_plan_labeled(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
                      const uint32_t *q_labels, const uint32_t *order, const uint32_t *po_pairs, int32_t npo,
                      uint32_t flags, const huge_mlp_t *model, huge_plan_t **out);
int huge_plan_free(huge_plan_t *p);
/*
 * Writes a one-line JSON description of the plan (operators, matching order, partial order,
 * estimated cost) into buf (host, len bytes, NUL-terminated, truncated if short).
 */
int huge_plan_describe(const huge_plan_t *p, char *buf, size_t len);
/* Host seconds the last huge_plan/huge_plan_ex spent, of which estimating cardinalities. */
int huge_plan_timing(const huge_plan_t *p, double *plan_s, double *estimate_s);
/*
 * The planner alone, on the host, with no graph and no GPU: the optimiser of Alg. 1 over
 * cardinalities the caller supplies, then the compilation of the chosen plan into operators
 * (Sec. 4.2: EXTEND with its partial-order bounds and injectivity checks, verify-only EXTEND
 * of Sec. 5.2, PUSH-JOIN with its key and cross-side filters). For inspecting and testing plans
 * and for planning with an estimator of one's own. With HUGE_PLAN_DIRECTED the query edges are
 * arcs and every step that reads a vertex's in-list lists "dirs" (1 = in-list) beside "ext".
 *  - nq, q_edges, mq, order, po_pairs, npo, flags: as huge_plan (HUGE_PLAN_LEARNED is rejected).
 *  - card (host, 2^nq doubles) or NULL when an order is given: card[mask] = the estimate of
 *    |R(q')| for the sub-query q' induced by the vertex set `mask` (bit v = query vertex v);
 *    read only for connected masks of two or more vertices.
 *  - edges_g: |E_G|, the pull term of an EXTEND in Alg. 1.
 *  - buf (host, len bytes): the plan as huge_plan_describe writes it ("how" is "given" or
 *    "offline"); a PUSH-JOIN plan adds "join_spec": lkey/rkey (key columns of each side, in the
 *    side's own vertex numbering = rank of the global id among the side's vertices),
 *    nonkey_l/nonkey_r, lr_l/lr_r (f_l[lr_l[i]] < f_r[lr_r[i]]), rl_r/rl_l
 *    (f_r[rl_r[i]] < f_l[rl_l[i]]), out_col_l/out_col_r (output column of each side column,
 *    -1 for the right side's key columns).
 * Errors: as huge_plan; HUGE_ERANGE when buf is too short (nothing written).
 */
int huge_plan_offline(uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
                      const uint32_t *po_pairs, int32_t npo, uint32_t flags, const double *card,
                      double edges_g, char *buf, size_t len);
/*
 * As huge_plan_offline for a labelled query: q_labels (host, nq entries, HUGE_ANY_LABEL for
 * any) and the label ranges of the graph the plan is for (lstart, host, nlabels + 1 entries:
 * label L owns the ids [lstart[L], lstart[L+1]), as huge_graph_label_ranges reports them). The
 * description then gives a labelled root's range as "root" and each labelled EXTEND's as "ids".
 */
int huge_plan_offline_labeled(uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *q_labels,
                              const uint32_t *lstart, uint32_t nlabels, const uint32_t *order,
                              const uint32_t *po_pairs, int32_t npo, uint32_t flags, const double *card,
                              double edges_g, char *buf, size_t len);

/* ======================================================================================= */
/* Enumerate                                                                               */
/* ======================================================================================= */

/*
 * Runs the plan on its graph (Sec. 4-5): SCAN of the first edge, PULL-EXTEND steps (and a
 * PUSH-JOIN if the plan has one), SINK. mode HUGE_COUNT writes the number of matches to
 * *out_count (host); HUGE_LIST also streams every match into `sink` (required then).
 * mem_bound_bytes bounds the device bytes held for intermediate partial matches (Sec. 5.2,
 * Thm. 5.3); it must cover at least one 32-row batch per level per resident warp, else
 * HUGE_ENOMEM. Errors: HUGE_ENOMEM, HUGE_EOVERFLOW, HUGE_ETIMEOUT, HUGE_ERANGE, HUGE_ECUDA.
 */
int huge_enumerate(const huge_plan_t *p, int mode, uint64_t mem_bound_bytes,
                   const huge_sink_t *sink, void *stream, int64_t *out_count);
/* As huge_enumerate, with options (root range or list, flags) and statistics (may be NULL). */
int huge_enumerate_ex(const huge_plan_t *p, int mode, uint64_t mem_bound_bytes,
                      const huge_sink_t *sink, void *stream, const huge_enum_opts_t *opts,
                      int64_t *out_count, huge_stats_t *stats);

/*
 * Batched form: counts nplans queries over the same graph in ONE persistent launch whose
 * warps take (query, root chunk) tasks from one device queue and steal work from each other.
 * Only EXTEND-chain plans are accepted (a plan with a PUSH-JOIN returns HUGE_EINVAL).
 * out_counts (host, nplans) receives each query's exact count.
 */
int huge_enumerate_batch(const huge_plan_t *const *plans, uint32_t nplans,
                         uint64_t mem_bound_bytes, void *stream, int64_t *out_counts,
                         huge_stats_t *stats);
/*
 * As huge_enumerate_batch, with options per plan (opts: host array of nplans entries, or
 * NULL): each plan's roots (roots/nroots, or root_begin/root_end), rows per level (level_cap)
 * and intersection variant are its own; flags and time_limit_ms apply to the whole launch (any
 * plan's HUGE_EF_* flag, the largest limit). The (query, root chunk) tasks of all plans are
 * queued heaviest first by estimated work (root weight 1 + degree times the plan's estimated
 * cost per unit weight), so the queries interleave. level_rows (optional, host, nplans x 16):
 * each plan's partial matches after each operator ([l] for operator l, the last operator's entry
 * holding the count, as huge_stats_t's level_rows from 1 on; unused entries 0). stats
 * (optional) sums over the batch.
 */
int huge_enumerate_batch_ex(const huge_plan_t *const *plans, uint32_t nplans, uint64_t mem_bound_bytes,
                            void *stream, const huge_enum_opts_t *opts, int64_t *out_counts,
                            int64_t *level_rows, huge_stats_t *stats);

/*
 * Autotuner: times candidate settings (rows per level per warp, root chunk size, the merge
 * variant of the last operator) for the given plans on the GPU and stores the fastest in each
 * plan; later enumerations of those plans use them. Then, while the budget lasts, it times the
 * graph's hub-bitmap degree threshold at half and twice its value and keeps the fastest
 * bitmaps on the graph (a setting of the graph, shared by all its plans). budget_ms caps the
 * device time spent. Writes the chosen level_cap and chunk_roots (host, may be NULL).
 */
int huge_autotune(huge_plan_t *const *plans, uint32_t nplans, uint64_t mem_bound_bytes,
                  double budget_ms, void *stream, uint32_t *level_cap, uint32_t *chunk_roots);

/* ======================================================================================= */
/* Learned cardinality estimator                                                           */
/* ======================================================================================= */

/*
 * A 3-layer perceptron 64 -> 128 -> 128 -> 1 (ReLU) that predicts log(1 + |R(q')|) for a
 * sub-query q' on a data graph, standing in for the cardinality estimate of Alg. 1 (its
 * cardinality term and the join costs) when plans are built with HUGE_PLAN_LEARNED.
 * Parameters are fp32 masters (layout: W1[128][64], b1[128], W2[128][128], b2[128], w3[128],
 * b3[1]; huge_mlp_num_params() entries), used in bf16 on the tensor cores with fp32
 * accumulation; inputs are standardised by per-feature mean mu[64] and scale sd[64] before
 * the first layer.
 * x: device float[rows][64]; y, t: device float[rows]; grad: device float[num_params].
 */
uint32_t huge_mlp_num_params(void);
int huge_mlp_create(uint64_t seed, huge_mlp_t **out);
int huge_mlp_free(huge_mlp_t *m);
/* host arrays; any of them may be NULL to leave it unchanged (resets the optimiser state) */
int huge_mlp_set_params(huge_mlp_t *m, const float *params, const float *mu, const float *sd);
int huge_mlp_get_params(const huge_mlp_t *m, float *params, float *mu, float *sd);
int huge_mlp_forward(const huge_mlp_t *m, const float *x, uint32_t rows, float *y, void *stream);
/* gradient of the loss 0.5 * mean((y - t)^2) at the current parameters; *loss on the host */
int huge_mlp_loss_grad(const huge_mlp_t *m, const float *x, const float *t, uint32_t rows, float *grad,
                       float *loss, void *stream);
/* Adam over `epochs` passes of minibatches of batch_rows rows (in the given order) */
int huge_mlp_train(huge_mlp_t *m, const float *x, const float *t, uint32_t rows, uint32_t epochs,
                   uint32_t batch_rows, float lr, float *final_loss, void *stream);
/*
 * The 64 estimator features of the sub-query of q induced by the vertex set `mask` (bit v =
 * query vertex v), with the transitive closure of the partial order (po as in huge_plan) inside
 * it, on graph g: graph statistics (sizes, degree moments and quantiles) and the sub-query's
 * shape (size, edges, partial-order pairs, triangles, wedges, 4-cycles, sorted degrees, ...).
 * out: host float[64].
 */
int huge_plan_features(const huge_graph_t *g, uint32_t nq, const uint32_t *q_edges, uint32_t mq,
                       const uint32_t *po_pairs, int32_t npo, uint32_t mask, float *out);

/*
 * Features of (plan, root) pairs for a learned model of per-root work, used to pre-partition
 * root vertices into balanced work (huge_enum_opts_t.root_weights): the 64 estimator features
 * of the plan's whole query (as huge_plan_features) with slots 46-56 replaced by statistics of
 * each root's neighbourhood computed on the device (log degree, log upward degree, log sums and
 * maximum of neighbour degrees, log two-hop upward size, relative id). roots: host, nroots ids
 * of the plan's graph (library ids); out: host float[nroots][64]. Undirected graphs only.
 * Errors: HUGE_EINVAL, HUGE_ENOMEM, HUGE_ECUDA.
 */
int huge_root_features(const huge_plan_t *p, const uint32_t *roots, uint64_t nroots, float *out);

/*
 * Allocation-free COUNT (the paper has no counterpart; this is an integration convenience).
 *
 * For callers that cannot call cudaMalloc: programs whose device memory is owned by another
 * allocator or fixed at start-up (a serving process that reserves its whole budget once, a
 * framework whose caching allocator must not see foreign allocations, an embedded user with a
 * hard memory limit), or that must not trigger the driver's allocation paths in steady state.
 * The caller passes the graph already on the device: d_offsets (uint32[n + 1], offsets[n] =
 * nnz) and d_adj (uint32[nnz]) in the CSR form huge_graph_load accepts (sorted, symmetric, no
 * self-loops, ids < n), used as given (no relabelling, no validation). Query, order (NULL: a
 * connected order chosen by the library) and partial order (npo = -1: automatic) follow
 * huge_plan; the count goes to *out_count (host).
 *
 * All scratch lives in one static device array of 32 MiB inside the library (every GPU that
 * loads the library holds it until the process exits). The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress with the device current) and caches it;
 * make that first call before any stream capture. Do not use this entry point on a device after
 * cudaDeviceReset: the cached address would then be stale. Every call re-initialises the parts of the
 * array that must start at zero; all calls share the one array, so calls whose kernels overlap
 * on the GPU (different streams or threads) race and must be serialised by the caller.
 * Nothing is allocated or freed. Errors: HUGE_EINVAL (arguments), HUGE_ENOMEM (the query's
 * minimum of 32 rows per level per warp does not fit in the 32 MiB array), HUGE_ETIMEOUT,
 * HUGE_EOVERFLOW, HUGE_ECUDA.
 */
int huge_count_noalloc(const uint32_t *d_offsets, const uint32_t *d_adj, uint32_t n, uint64_t nnz,
                       uint32_t nq, const uint32_t *q_edges, uint32_t mq, const uint32_t *order,
                       const uint32_t *po_pairs, int32_t npo, void *stream, int64_t *out_count);

/*
 * Caller allocator hook (ownership of device memory). Every device buffer the library keeps
 * (graph CSR, hub bitmaps, enumeration and join workspaces, MLP parameters) is obtained with
 * alloc(ctx, bytes, device) and returned with free(ctx, ptr, device) on the same allocator that
 * made it, even if the hook changes in between (device: the one current at allocation); alloc returns NULL on failure (the call then
 * fails with HUGE_ENOMEM). Both NULL restores cudaMalloc / cudaFree. The PyTorch binding sets
 * a hook onto torch's caching allocator so that PyTorch owns those bytes. The library calls
 * the hook only from the thread that called into it, between stream synchronisations.
 * huge_count_noalloc never allocates and never calls it.
 */
typedef void *(*huge_alloc_fn)(void *ctx, size_t bytes, int device);
typedef void (*huge_free_fn)(void *ctx, void *ptr, int device);
int huge_set_allocator(huge_alloc_fn alloc, huge_free_fn free_fn, void *ctx);

/* Thread-local message describing the last error of this thread ("" if none). */
const char *huge_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HUGE_H */
