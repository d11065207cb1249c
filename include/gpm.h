/*
 * gpm.h — C ABI of the GB300 pattern-aware subgraph enumeration library.
 *
 * The library counts and lists the matches of a small pattern P in a large
 * undirected data graph G (G2Miner, arXiv 2112.09761).  A match is one
 * distinct subgraph of G isomorphic to P, found once (completeness and
 * uniqueness, Section 2.1; symmetry order, Section 2.2).  Vertex-induced
 * matches require P's non-edges to be non-edges of G; edge-induced matches do
 * not (Section 2.1).  For cliques the two coincide.
 *
 * Everything on the enumeration path runs in this library's own CUDA kernels
 * for sm_103a: loading and validating the CSR, orienting it, building the root
 * task list, the warp-cooperative DFS with set intersection / difference /
 * bounding, the reductions and the listing output.  There is no CPU fallback:
 * a process without a usable GPU gets GPM_E_CUDA.
 *
 * Conventions
 *   - Every call returns a gpm_status.  On error nothing is written to the
 *     outputs and gpm_last_error() (thread-local) describes the failure.
 *   - Handles (gpm_graph, gpm_plan_t) are opaque and library-owned.
 *   - `stream` arguments are cudaStream_t values passed as void*; NULL is the
 *     legacy default stream.  Calls that return host results synchronise that
 *     stream before returning.
 *   - Vertex IDs are uint32; counts are uint64; all arithmetic is integer.
 *   - A handle may be used by one host thread at a time.
 */
#ifndef GPM_H_
#define GPM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gpm_status {
  GPM_OK = 0,
  GPM_E_INVALID_ARG = 1,         /* NULL pointer, bad size, bad flag combination */
  GPM_E_UNSORTED = 2,            /* a neighbour list is not strictly ascending */
  GPM_E_SELF_LOOP = 3,           /* v appears in N(v) */
  GPM_E_DUPLICATE = 4,           /* a neighbour appears twice in one list */
  GPM_E_ASYMMETRIC = 5,          /* u in N(v) but v not in N(u) */
  GPM_E_OOM = 6,                 /* a device or pinned-host allocation failed */
  GPM_E_UNSUPPORTED_PATTERN = 7, /* the pattern matches no plan family */
  GPM_E_CAPACITY = 8,            /* listing output truncated (n_total still valid) */
  GPM_E_TIMEOUT = 9,             /* a bounded device-side wait gave up */
  GPM_E_CUDA = 10,               /* CUDA runtime error (no device, launch failure, ...) */
  GPM_E_RANGE = 11               /* an ID or offset outside [0, n) / [0, nnz] */
} gpm_status;

/* ------------------------------------------------------------ patterns */

/* A pattern: k <= 8 vertices (0..k-1) and an undirected edge list.  The
 * pattern must be connected.  (Section 4.1: patterns are given explicitly by
 * their edge list, or by helpers such as generateClique.) */
typedef struct gpm_pattern {
  uint32_t k;
  uint32_t n_edges;
  uint8_t edges[28][2];
} gpm_pattern;

/* Fill *out with a named pattern.  Names: "triangle", "<k>-clique" (k=3..8),
 * "diamond", "4-cycle", "tailed-triangle", "3-star", "4-path", "wedge".
 * The edge list is given in the library's matching order, i.e. the order in
 * which gpm_list() writes the k vertices of each match:
 *   k-clique         v1..vk in the degree-orientation order of the clique
 *   diamond          (v1,v2) the chord, v3 > v4 the other two
 *   4-cycle          v1 = the largest ID, cycle v1-v2-v3-v4-v1, v2 > v4
 *   tailed-triangle  v1 the degree-3 vertex, triangle v1 v2 v3 (v3 < v2), tail v4
 *   3-star           centre v1, leaves v2 > v3 > v4
 *   4-path           path v3-v1-v2-v4, middle edge v1 > v2
 *   wedge            centre v1, ends v2 > v3
 * Returns GPM_E_UNSUPPORTED_PATTERN for an unknown name. */
gpm_status gpm_pattern_named(const char* name, gpm_pattern* out);

/* -------------------------------------------------------------- graphs */

typedef struct gpm_graph gpm_graph;

#define GPM_DEVICE_PTRS 1u   /* offsets / nbrs are device pointers (else host) */
#define GPM_BORROW 2u        /* keep the caller's device arrays instead of copying;
                                needs GPM_DEVICE_PTRS and 64-bit offsets; the caller
                                keeps them alive and unchanged until gpm_graph_free */
#define GPM_SKIP_VALIDATE 4u /* trust the input (no sortedness / symmetry check) */
#define GPM_RELABEL 8u       /* rename the vertices by degree order (see below) */

/*
 * Load an undirected data graph in CSR form (Section 4.2 graph loader).
 *   offsets      n+1 row offsets, int32 (offsets_is_64 = 0) or int64 (= 1);
 *                offsets[0] = 0, non-decreasing, offsets[n] = nnz
 *   nbrs         nnz uint32 neighbour IDs; row v is nbrs[offsets[v] ..
 *                offsets[v+1]); each row strictly ascending, no v in N(v),
 *                and u in N(v) iff v in N(u) (both directions present)
 *   n, nnz       vertices and directed entries (nnz = 2|E|); n < 2^32 - 1
 *   flags        GPM_DEVICE_PTRS | GPM_BORROW | GPM_SKIP_VALIDATE | GPM_RELABEL
 *   stream       stream for the copies and the validation kernels
 * The library copies the arrays to device memory it owns (int64 offsets),
 * computes degrees and the maximum degree, and (unless skipped) validates the
 * input on the GPU, returning GPM_E_UNSORTED / _SELF_LOOP / _DUPLICATE /
 * _ASYMMETRIC / _RANGE for the first violation class found.
 * Derived structures (degree-oriented DAG, root task lists) are built on the
 * device the first time a plan needs them and cached with the graph.
 * GPM_RELABEL (Section 4.2 preprocessing: sorting and renaming the vertices by
 * degree) renames the validated graph on the device: new vertex i is the
 * vertex of rank i in ascending (degree, id) order, rows re-sorted.  Counts
 * do not change; gpm_list translates its matches back to the caller's IDs.
 * The renamed arrays are owned by the library even under GPM_BORROW (the
 * caller's arrays are then only read during this call).  Renaming needs
 * 8 B x (nnz rounded up to a power of two) of temporary device memory.
 */
gpm_status gpm_load_csr(const void* offsets, int offsets_is_64, const uint32_t* nbrs, uint32_t n,
                        uint64_t nnz, uint32_t flags, void* stream, gpm_graph** out);

/* Input information extracted while loading (Section 4.2: |V|, |E|, max
 * degree).  Any output pointer may be NULL.  max_out_degree is the maximum
 * out-degree of the degree-oriented DAG (0 until a clique plan built it). */
gpm_status gpm_graph_info(const gpm_graph* g, uint32_t* n, uint64_t* n_edges, uint32_t* max_degree,
                          uint32_t* max_out_degree);

/* Copy the graph as the library holds it to host memory: offsets int64[n+1],
 * nbrs uint32[nnz] and, if perm is not NULL, perm uint32[n] = the caller's ID
 * of every vertex (the identity unless loaded with GPM_RELABEL).  Synchronises
 * `stream`. */
gpm_status gpm_graph_export(const gpm_graph* g, int64_t* offsets, uint32_t* nbrs, uint32_t* perm,
                            void* stream);

/* Release the graph and everything cached with it.  NULL is ignored. */
void gpm_graph_free(gpm_graph* g);

/* --------------------------------------------------------------- plans */

typedef struct gpm_plan_s gpm_plan_t;

#define GPM_COUNT 0
#define GPM_LIST 1

/* Execution knobs.  Zero means "choose automatically" for every field. */
typedef struct gpm_plan_opts {
  uint32_t warps_per_block;  /* warps per CTA of the enumeration kernel */
  uint32_t blocks_per_sm;    /* resident CTAs per SM of the persistent grid */
  uint32_t chunk;            /* root tasks taken per grab from the task queue */
  uint32_t bsearch_ratio;    /* |B| >= ratio * |A| selects binary search over merge */
  uint32_t no_count_only;    /* 1 = enumerate even where a counting-only form exists */
  uint32_t collect_stats;    /* 1 = count algorithmic bytes / set operations (slower) */
  uint32_t no_lgs;           /* 1 = cliques (and batched 4-cliques) without local graph
                                search (sorted sets only) */
  uint32_t generic_plan;     /* 1 = run the generic interpreter even for a named family */
  uint32_t vertex_parallel;  /* 1 = root tasks are vertices (Section 5.1 vertex parallelism):
                                a warp takes a vertex v1 and walks its root pairs (v1, v2)
                                from its row, no task list Omega is built, task ranges are
                                vertex ranges; cliques then use the sorted-set kernel */
} gpm_plan_opts;

/*
 * Build an execution plan (Section 4.2 pattern analyzer, Section 7.2 memory
 * management) for counting or listing `pattern` in `g`:
 *   induced   0 = edge-induced, 1 = vertex-induced
 *   mode      GPM_COUNT or GPM_LIST
 *   opts      NULL for automatic choices
 * The pattern is identified up to isomorphism with one of the named families
 * (k-clique up to k = 8, diamond, 4-cycle, tailed-triangle, 3-star, 4-path,
 * wedge), which have hand-written plans.  Any other connected pattern of 3 to
 * 8 vertices (or any pattern with opts->generic_plan) gets a search plan from
 * the pattern analyzer: the matching order with the least estimated
 * neighbour-list reading over all valid orders, and a symmetry order built
 * along it from the pattern's automorphisms (each vertex the largest of its
 * orbit under the automorphisms fixing the earlier ones), run by the generic
 * interpreter.  Disconnected patterns, or fewer than 3 or more than 8
 * vertices, return GPM_E_UNSUPPORTED_PATTERN.  The plan fixes the matching
 * order, the symmetry order, the root task list Omega (reduced to v1 > v2 when
 * the symmetry order allows, Section 7.2 (2)), the per-warp DFS buffers
 * (Section 7.2 (3)) and the grid; it builds the DAG / task lists on the device
 * if the graph has not cached them yet.  Listings write each match as k
 * uint32, entry i being the data vertex matched to pattern vertex i for
 * generic plans and the plan's matching order for the named families.
 */
gpm_status gpm_plan(gpm_graph* g, const gpm_pattern* pattern, int induced, int mode,
                    const gpm_plan_opts* opts, void* stream, gpm_plan_t** out);

/* Number of root tasks |Omega| of the plan: DAG arcs for cliques (listed by
 * source then destination ID), pairs v1 > v2 for diamond / 4-cycle / 4-path
 * (by v1 then v2), and all directed CSR entries for tailed-triangle / 3-star /
 * wedge (CSR order); generic plans use pairs v1 > v2 when their symmetry order
 * holds v0 > v1, else all directed entries.  This order defines the task
 * ranges of gpm_count_range.  With opts->vertex_parallel the tasks are the n
 * vertices instead (vertex v roots the pairs of its row). */
gpm_status gpm_plan_info(const gpm_plan_t* p, uint64_t* n_tasks, uint32_t* k);

/* The plan as text (NUL-terminated, at most len bytes with the NUL): its
 * family and, for generic plans, the matching order as pattern vertices
 * ("order: u1 u0 u2 ..."), the symmetry order over matching positions
 * ("symmetry: v0>v1 v2>v3", vi = the data vertex at position i), the root
 * task list and the induced mode.  GPM_E_CAPACITY if the text was cut. */
gpm_status gpm_plan_describe(const gpm_plan_t* p, char* buf, size_t len);

/* Number of kernels the library enqueues for one evaluation of the plan
 * (count, non-empty task range or listing); memsets and copies are not
 * counted. */
gpm_status gpm_plan_launches(const gpm_plan_t* p, uint32_t* n);

/* The search plan gpm_plan would choose for `pattern` on a graph of n
 * vertices and nnz directed entries (the cost model's inputs), as the same
 * text, without a graph or a GPU: host-side pattern analysis only.  generic =
 * 1 analyses named families as gpm_plan does with opts->generic_plan. */
gpm_status gpm_pattern_describe(const gpm_pattern* pattern, int induced, uint32_t n, uint64_t nnz,
                                int generic, char* buf, size_t len);

/* Count all matches (Section 4.1 count()).  *out_count is a host uint64.
 * Synchronises `stream`. */
gpm_status gpm_count(gpm_plan_t* p, uint64_t* out_count, void* stream);

/* Count the matches rooted at tasks [task_lo, task_hi) of Omega (clamped to
 * |Omega|).  Summing disjoint ranges gives gpm_count's result. */
gpm_status gpm_count_range(gpm_plan_t* p, uint64_t task_lo, uint64_t task_hi, uint64_t* out_count,
                           void* stream);

/*
 * List matches (Section 4.1 list()).  Writes at most `capacity` matches of k
 * uint32 each (the plan's matching order, see gpm_pattern_named) to the
 * DEVICE buffer out_dev (capacity * k uint32), in an unspecified order.
 * *n_written = min(total, capacity), *n_total = all matches.  Returns
 * GPM_E_CAPACITY (with both outputs valid) when the buffer was too small.
 * The plan must have been built with GPM_LIST.  Synchronises `stream`.
 */
gpm_status gpm_list(gpm_plan_t* p, uint32_t* out_dev, uint64_t capacity, uint64_t* n_written,
                    uint64_t* n_total, void* stream);

/*
 * Statistics of the plan's last gpm_count / gpm_count_range / gpm_list call,
 * available when the plan was built with collect_stats = 1 (GPM_E_INVALID_ARG
 * otherwise).  All are integers independent of the schedule.
 *   alg_bytes  sum over every sorted-set operation A∘B (Section 6.1) of
 *              4 * (min(|A|,|B|) + min(max(|A|,|B|), min(|A|,|B|) *
 *              ceil(log2(max(|A|,|B|) + 1)))) operand bytes (the cheaper of a
 *              merge and a binary search), 16 B of list offsets and 4 B per
 *              written element, plus 8 B per root task;
 *   set_ops    number of sorted-set operations of the sorted-set kernels;
 *   word_ops   bitmap word operations of the local graph search (Section
 *              5.4 (2), Section 6.2): one per 32-bit AND(+POPC) of two bitmap
 *              rows and one per single-bit membership test.
 * Any output pointer may be NULL.
 */
gpm_status gpm_plan_stats(const gpm_plan_t* p, uint64_t* alg_bytes, uint64_t* set_ops,
                          uint64_t* word_ops);

/* Release the plan.  NULL is ignored. */
void gpm_plan_free(gpm_plan_t* p);

/* -------------------------------------------------------- motifs, batches */

/*
 * Vertex-induced k-motif counts of one graph (Section 2.1 k-MC; Section 5.3
 * multi-pattern fission; Section 5.4 (1) counting-only pruning by pattern
 * decomposition).  k = 3: out[0..1] = {wedge, triangle}.  k = 4: out[0..5] =
 * {4-path, 3-star, 4-cycle, tailed-triangle, diamond, 4-clique}.  Only
 * connected patterns are counted.  `out` is host memory.  Equivalent to a
 * batch of one graph; synchronises `stream`.
 */
gpm_status gpm_motif_count(gpm_graph* g, uint32_t k, uint64_t* out, void* stream);

typedef struct gpm_batch_s gpm_batch_t;

/*
 * Prepare k-motif counting (k = 3 or 4) over n_graphs resident graphs, run as
 * one persistent launch per kernel family over a device-side queue of
 * (graph, root) tasks spanning all graphs, captured once into a CUDA graph.
 * Builds each graph's DAG and task lists if not cached.  With opts->chunk,
 * opts->bsearch_ratio and opts->warps_per_block all zero, an autotuner times
 * candidate task-chunk sizes, intersection thresholds and CTA shapes on the
 * batch itself and keeps the fastest; nonzero fields fix them.  For k = 4 the
 * 4-cliques of all graphs are counted by local graph search (bitmap local
 * graphs, roots of every graph sorted into out-degree classes once here)
 * unless opts->no_lgs is set, in which case the sorted-set kernel counts
 * them; both give the same counts.  The graphs must outlive the batch.  Returns GPM_E_INVALID_ARG for k not in {3, 4} or
 * n_graphs = 0.
 */
gpm_status gpm_batch_create(gpm_graph* const* graphs, uint32_t n_graphs, uint32_t k,
                            const gpm_plan_opts* opts, void* stream, gpm_batch_t** out);

/* Run the batch: out is host uint64[n_graphs][2 or 6], per graph the counts
 * in gpm_motif_count's order.  Synchronises `stream`. */
gpm_status gpm_batch_count(gpm_batch_t* b, uint64_t* out, void* stream);

/* Chosen configuration of a batch (after autotuning): task chunk,
 * intersection threshold, warps per CTA of the per-edge kernels. */
gpm_status gpm_batch_info(const gpm_batch_t* b, uint32_t* chunk, uint32_t* bsearch_ratio,
                          uint32_t* warps_per_block);

/* Release the batch (not its graphs).  NULL is ignored. */
void gpm_batch_free(gpm_batch_t* b);

/* ---------------------------------------------------------------- serving */

typedef struct gpm_server_s gpm_server_t;

/*
 * A query server over resident graphs with continuous batching (a serving
 * extension of Section 7.2 (3) adaptive buffering: a query's device memory is
 * its plan's DFS buffers, counters and root lists).  Up to max_inflight
 * queries (1..256) run concurrently on their own streams; a pending query is
 * admitted, in arrival order, when a slot is free and its memory fits in
 * mem_budget bytes (a query that does not fit yet is passed over by smaller
 * ones behind it; one that exceeds the whole budget runs alone when the
 * server is otherwise idle).  Plans are built on first use and cached per
 * (graph, pattern, induced).  A scheduler thread polls CUDA events: no
 * device-side waits.  The graphs must outlive the server and must not be used
 * through other calls while the server may build plans on them.
 */
gpm_status gpm_server_create(size_t mem_budget, uint32_t max_inflight, gpm_server_t** out);

/* Submit a count query; *ticket identifies it.  Thread-safe. */
gpm_status gpm_server_submit(gpm_server_t* s, gpm_graph* g, const gpm_pattern* pattern,
                             int induced, uint64_t* ticket);

/* Non-blocking: *done = 1 once the query finished; then *count and
 * *latency_s (submission to completion, seconds) are written (either may be
 * NULL) and the query's own status is returned. */
gpm_status gpm_server_poll(gpm_server_t* s, uint64_t ticket, int* done, uint64_t* count,
                           double* latency_s);

/* Block until the query finished or timeout_s elapsed (GPM_E_TIMEOUT). */
gpm_status gpm_server_wait(gpm_server_t* s, uint64_t ticket, double timeout_s, uint64_t* count,
                           double* latency_s);

/* Counters: completed queries, pending queries, the largest number of
 * queries in flight at once, device bytes admitted right now. */
gpm_status gpm_server_stats(gpm_server_t* s, uint64_t* completed, uint64_t* pending,
                            uint64_t* peak_inflight, size_t* bytes_in_use);

/* Stop the scheduler after in-flight work drains, free plans and streams.
 * Pending queries are dropped.  NULL is ignored. */
void gpm_server_free(gpm_server_t* s);

/* ------------------------------------------------- allocation-free count */

/*
 * Triangle count of an undirected graph whose CSR is already in device memory,
 * for callers that must not allocate device memory (loops where cudaMalloc /
 * cudaFree could synchronise the device and stall other streams; plug-ins
 * whose host application owns all device memory; processes that reserve all
 * their device memory up front).  The paper has no counterpart to this entry
 * point: it is a service of this library.
 *   offsets_dev  int64[n+1] device row offsets; nbrs_dev uint32 device
 *                neighbour lists (sorted ascending, both directions, no loops
 *                or duplicates; not validated here; may be NULL when the graph
 *                has no edges)
 *   count_dev    device uint64 that receives the count (written last)
 *   stream       enqueued on `stream`; the call does not synchronise it
 * No memory is allocated: all working memory is one fixed 1 MiB device array
 * in the library, so n may be at most 131,069 (GPM_E_INVALID_ARG beyond).
 * The first call on a device looks the array up for that device; make that
 * first call before any stream capture.  Calls share the array: calls that
 * overlap on the GPU (for example on two streams) race; serialise them.
 */
gpm_status gpm_count_triangles_noalloc(const int64_t* offsets_dev, const uint32_t* nbrs_dev,
                                       uint32_t n, uint64_t* count_dev, void* stream);

/* ------------------------------------------------------------- errors */

/* Description of the last error on this host thread ("" if none). */
const char* gpm_last_error(void);

/* Library version string. */
const char* gpm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GPM_H_ */
