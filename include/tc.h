/*
 * tc.h — C ABI of the GB300 triangle-centrality library (libtc_gb300.so).
 *
 * Triangle centrality (P. Burkhardt, "Triangle Centrality", Definition 1):
 *
 *   TC(v) = ( ⅓ Σ_{u ∈ N△[v]} △(u) + Σ_{w ∈ N(v) \ N△(v)} △(w) ) / △(G)
 *
 * where △(v) is the number of triangles on v, △(G) the number in G,
 * N△(v) = { u ∈ N(v) : N(u) ∩ N(v) ≠ ∅ } the triangle neighbours of v and
 * N△[v] = {v} ∪ N△(v) (section "Notation").  The library computes it in
 * the four steps of the paper's elementary algorithm (section "Algorithm",
 * figure "Triangle centrality elementary algorithm"; Algorithm 2):
 *
 *   tc_build_csr   simple undirected graph from a pair list, degree order
 *                  π (degree, then label) and orientation N_H / N_L
 *                  (section "Notation"; Lemma 1's partition of N(v));
 *   tc_count       △(v), △(G) and the in-a-triangle flag of every edge
 *                  (steps 1 and 2; Procedure 1 and its alternative in
 *                  the appendix "Alternative Triangle Neighbor Algorithm");
 *   tc_centrality  the exact integer numerator
 *                      numer(v) = Σ_{u∈N△[v]} △(u) + 3 Σ_{w∈N(v)\N△(v)} △(w)
 *                                = 3 · △(G) · TC(v)
 *                  and one binary64 division TC(v) = numer(v) / (3△(G)),
 *                  rounded to nearest-even (step 3; Algorithm 2, whose
 *                  (x/3 + y)/△(G) is the same quotient computed exactly).
 *
 * Conventions for every entry point:
 *   - Vertex ids are 0-based in [0, n) (the paper labels 1..n).
 *   - Pointers named d_* are device pointers, h_* host pointers.  Device
 *     outputs are caller-allocated and caller-owned; the library never
 *     frees them.  A tc_graph owns its own device memory until
 *     tc_graph_free.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All
 *     device work of a call is ordered on that stream.  A call that returns
 *     a host scalar synchronises the stream before returning.
 *   - No exception crosses the ABI.  On a negative status, outputs are
 *     unspecified; *out pointers are set to NULL.
 *   - One tc_graph must not be used by two calls at the same time; calls on
 *     different graphs are independent.
 *   - All integer results (counts, flags, numerators) are exact.
 */
#ifndef TC_GB300_H
#define TC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tc_stream;   /* the same type as cudaStream_t */
typedef struct tc_graph tc_graph;        /* opaque */

typedef enum {
    TC_OK = 0,
    TC_NO_TRIANGLES = 1,        /* warning: △(G) = 0; TC is NaN everywhere   */
    TC_ERR_INVALID_ARG = -1,    /* bad pointer, size or vertex id             */
    TC_ERR_OUT_OF_MEMORY = -2,  /* device or host allocation failed          */
    TC_ERR_CUDA = -3,           /* any other CUDA runtime error               */
    TC_ERR_OVERFLOW = -4,       /* 3·△(G) does not fit in 64 bits             */
    TC_ERR_TIMEOUT = -5,        /* a bounded device-side wait gave up         */
    TC_ERR_STATE = -6,          /* call order violated (e.g. no tc_count yet) */
    TC_ERR_BOUNDS = -7          /* bounds-checked builds only: a kernel's index
                                   check failed (the access was skipped)      */
} tc_status;

/* tc_build_csr flags */
#define TC_IN_DEVICE 1u   /* src/dst are device pointers (else pageable or pinned host) */
#define TC_IDS_INT32 2u   /* src/dst hold int32_t ids (else int64_t)                     */

/* Intersection strategies (tc_set_strategy).  AUTO lets the planner choose
 * per work item by degree bucket; the others force one strategy for every
 * item (used to test each strategy alone).                                   */
#define TC_STRATEGY_AUTO    0
#define TC_STRATEGY_BSEARCH 1   /* binary search of each streamed id in N_H(v) staged in shared memory */
#define TC_STRATEGY_MERGE   2   /* warp-cooperative merge-path intersection of two sorted lists         */
#define TC_STRATEGY_BITMAP  3   /* N_H(v) as a shared-memory bitmap over its id window (falls back to
                                   BSEARCH for an item whose window does not fit)                       */
#define TC_STRATEGY_GLOBAL  4   /* binary search of N_H(v) in place in global memory (what lists too
                                   long for shared memory use under every other strategy)              */

/*
 * Build the simple undirected graph G from `num_pairs` pairs (src[i],
 * dst[i]) over vertices [0, n): pairs are symmetrised, self-loops and
 * duplicates dropped (the set-up of the paper's section "Comparison").
 * The graph is then relabelled by the degree order π of section "Notation"
 * (ascending degree, ties by label) and every adjacency row sorted, so that
 * the lower neighbours N_L(v) and the higher neighbours N_H(v) are the two
 * contiguous halves of row v; this is the partition of Lemma 1.
 *
 *   src, dst   num_pairs ids each; device pointers if flags & TC_IN_DEVICE,
 *              else host pointers (copied to the device inside the call);
 *              int32_t if flags & TC_IDS_INT32, else int64_t.  Read only.
 *   n          vertex count, 0 <= n <= 2^31 - 1.
 *   out        receives the new graph (owned by the caller, release with
 *              tc_graph_free), or NULL on error.
 * Errors: TC_ERR_INVALID_ARG for NULL pointers with num_pairs > 0, negative
 * sizes, n too large or any id outside [0, n); TC_ERR_OUT_OF_MEMORY;
 * TC_ERR_CUDA.  Synchronises `stream`.
 */
tc_status tc_build_csr(const void* src, const void* dst, int64_t num_pairs, int64_t n,
                       uint32_t flags, tc_stream stream, tc_graph** out);

/*
 * Steps 1-2 of the elementary algorithm: per-vertex triangle counts △(v),
 * the total △(G) and the in-a-triangle flag of every edge (u ∈ N△(v)).
 * Each triangle is found once, from the oriented edge joining its two
 * lowest-ordered vertices, by intersecting their higher neighbourhoods
 * (Procedure 1; appendix "Alternative Triangle Neighbor Algorithm").
 *
 *   d_tri        [n] uint64, caller labels: d_tri[v] = △(v).  May be NULL.
 *   d_edge_flag  [m] uint8, aligned with the canonical edge list of
 *                tc_graph_info: 1 if that edge lies in at least one
 *                triangle, else 0.  May be NULL.
 *   h_tri_total  receives △(G).  May be NULL.
 * The counts and flags are also kept inside the graph for tc_centrality.
 * Returns TC_OK, or TC_NO_TRIANGLES if △(G) = 0 (outputs still valid, all
 * zero).  Synchronises `stream`.
 */
tc_status tc_count(tc_graph* g, uint64_t* d_tri, uint8_t* d_edge_flag,
                   uint64_t* h_tri_total, tc_stream stream);

/*
 * Sharded count (steps 1-2 split across K shards: K GPUs, or K passes on
 * one).  Every triangle is found exactly once, by one work item of the
 * count (Procedure 1: at its middle vertex, from its lowest vertex), so the
 * work items can be dealt out: shard k of K counts the items k, k + K, ...
 * and returns the partial △(v) of the triangles it found and the flags of
 * their edges.  Summing the partial △(v) over the shards and OR-ing their
 * flags gives exactly what tc_count gives; tc_load_counts takes that result
 * back into a graph so that tc_centrality can follow.  Every shard must
 * hold the same graph (built from the same pairs).
 *
 *   shard, num_shards  0 <= shard < num_shards.
 *   d_tri        [n] uint64, caller labels: this shard's partial △(v).
 *   d_edge_flag  [m] uint8, canonical edge order: 1 where this shard found
 *                a triangle on the edge.
 *   h_tri_partial receives the triangles this shard found.
 * Any output may be NULL.  Leaves the graph without valid counts (call
 * tc_load_counts or tc_count before tc_centrality).  Synchronises `stream`.
 */
tc_status tc_count_shard(tc_graph* g, int shard, int num_shards, uint64_t* d_tri, uint8_t* d_edge_flag,
                         uint64_t* h_tri_partial, tc_stream stream);

/*
 * Loads complete counts — △(v) [n] uint64 in caller labels and the edge
 * flags [m] uint8 in canonical edge order, e.g. the sum and the OR of every
 * shard's tc_count_shard outputs — into g, sets △(G) = Σ △(v) / 3 and makes
 * g ready for tc_centrality.  Returns TC_ERR_INVALID_ARG if Σ △(v) is not a
 * multiple of 3 (the inputs cannot be complete counts), TC_NO_TRIANGLES if
 * △(G) = 0, else TC_OK; h_tri_total (may be NULL) receives △(G).
 * Synchronises `stream`.
 */
tc_status tc_load_counts(tc_graph* g, const uint64_t* d_tri, const uint8_t* d_edge_flag, uint64_t* h_tri_total,
                         tc_stream stream);

/*
 * Per-edge triangle counts t(u, v) = (A² ∘ A)(u, v), the number of
 * triangles on each edge (section "Notation": T = A² ∘ A, whose row sums
 * are 2△(v), section "Algebraic Form"), computed by the same pass as
 * tc_count: wherever tc_count marks an edge as lying in a triangle, this
 * call adds the number of triangles found there instead.
 *
 *   d_tri        [n] uint64, caller labels: △(v).  May be NULL.
 *   d_edge_tri   [m] uint32, aligned with the canonical edge list of
 *                tc_graph_info: t(u, v) of that edge.  May be NULL.
 *   h_tri_total  receives △(G) = Σ t(u, v) / 3.  May be NULL.
 * Also leaves the counts and edge flags (flag = t > 0) in the graph, so
 * tc_centrality may follow.  Takes 4 bytes per CSR entry (8 per edge) of
 * extra device memory, held by the graph until tc_graph_free.  Returns
 * TC_OK or TC_NO_TRIANGLES.  Synchronises `stream`.
 */
tc_status tc_edge_triangles(tc_graph* g, uint64_t* d_tri, uint32_t* d_edge_tri, uint64_t* h_tri_total,
                            tc_stream stream);

/*
 * Step 3: for every vertex the exact numerator
 *   numer(v) = △(v) + Σ_{u ∈ N(v)} (u ∈ N△(v) ? 1 : 3) · △(u)
 * (the core sum x plus three times the non-core sum y of Algorithm 2), and
 * TC(v) = numer(v) / (3△(G)) rounded once to nearest-even binary64.  Uses
 * the counts and flags of the most recent tc_count on g.
 *
 *   d_numer  [n] uint64, caller labels.  May be NULL.
 *   d_tc     [n] double, caller labels.  May be NULL.  NaN everywhere if
 *            △(G) = 0.
 *   h_den    receives the denominator 3△(G).  May be NULL.
 * Returns TC_OK, TC_NO_TRIANGLES, or TC_ERR_STATE if tc_count has not run
 * on g.  Does not synchronise `stream`.
 */
tc_status tc_centrality(tc_graph* g, uint64_t* d_numer, double* d_tc, uint64_t* h_den,
                        tc_stream stream);

/*
 * The division of step 3 on its own: d_tc[i] = d_numer[i] / den rounded to
 * nearest-even binary64, exact for every 64-bit numerator and denominator
 * (den = 0 gives NaN).  d_numer and d_tc are device arrays of n elements.
 * Does not synchronise `stream`.
 */
tc_status tc_divide(const uint64_t* d_numer, int64_t n, uint64_t den, double* d_tc,
                    tc_stream stream);

/*
 * The canonical edge list of g: m undirected edges (d_edge_u[i], d_edge_v[i])
 * with d_edge_u[i] < d_edge_v[i], caller labels, sorted by (u, v).  The
 * pointers stay owned by g and valid until tc_graph_free.  Any output
 * pointer may be NULL.
 */
tc_status tc_graph_info(const tc_graph* g, int64_t* n, int64_t* m,
                        const int32_t** d_edge_u, const int32_t** d_edge_v);

/*
 * Copies the canonical edge list into caller device buffers of m int32 each
 * (d_u[i] < d_v[i], caller labels, sorted by (u, v)); either may be NULL.
 * Ordered on `stream`; does not synchronise it.
 */
tc_status tc_copy_edges(const tc_graph* g, int32_t* d_u, int32_t* d_v, tc_stream stream);

/* Shape statistics of g, computed at build time (host values). */
typedef struct {
    int64_t n, m;
    int64_t max_degree;
    int64_t max_out_degree;      /* max |N_H(v)|                                        */
    double  sum_out_degree_sq;   /* Σ_v |N_H(v)|²                                       */
    double  wedges;              /* Σ_v C(|N_H(v)|, 2): ids streamed by the count step   */
    double  avg_degeneracy;      /* δ̄ = (1/m) Σ_{(v,u)∈E} min(d(v), d(u))              */
    int64_t items[5];            /* count-step work items per class: bitmap (small shared
                                    footprint), bitmap (large), warp, CTA list, thread
                                    (one thread per tiny vertex)                        */
    double  class_bytes[5];      /* algorithmic DRAM bytes of each class's kernel       */
    double  class_wedges[5];     /* ids streamed by each class                          */
    double  class_head[5];       /* head entries (lower neighbours) of each class       */
    double  count_bytes;         /* algorithmic DRAM bytes of the whole count step      */
    double  centrality_bytes;    /* algorithmic DRAM bytes of the gather + divide step  */
    int64_t core_vertices;       /* C of the dense core (0: none): the top C ranks,
                                    whose mutual triangles are counted edge by edge
                                    from bit-packed core rows; the counts above then
                                    leave that work out                                */
    double  core_words;          /* 32-bit row words ANDed by that pass per count
                                    (core edges x words per packed core row)          */
} tc_graph_stats;

tc_status tc_get_stats(const tc_graph* g, tc_graph_stats* out);

/*
 * Dense core of the count step (an implementation choice, no counterpart in
 * the paper; results never change).  Among the highest ranks of the degree
 * order (Lemma 1's orientation puts the hubs last) the adjacency is dense,
 * and every triangle whose lowest vertex is among the top C ranks lies there
 * entirely.  For such a core tc_count counts those triangles edge by edge:
 * on each core edge (x, y), T(x, y) = |N_c(x) ∩ N_c(y)| is the AND and
 * population count of the two bit-packed core rows — the matrix form
 * T = A² ∘ A of the section "Notation" restricted to the core, evaluated
 * only on its edges — and the sparse kernels skip those triangles.
 *
 * Process-wide setting read by later tc_build_csr calls: c = -1 (default)
 * lets each build choose C in {4096, 8192, 16384, 32768} when the bit-packed
 * pass is expected to be faster than streaming the core's rows (else no
 * core); c = 0 never; 0 < c <= 32768 uses the top min(c, n) ranks.  Batches
 * never use a core.  A count with a core holds C·W·6 + 8·C bytes of device
 * memory while it runs, W = ⌈C/32⌉ rounded up to 128, 256, 512 or 1024
 * (48 MB at C = 16384).  Returns TC_ERR_INVALID_ARG for c < -1 or
 * c > 32768.
 */
tc_status tc_set_dense_core(long long c);

/* Force one intersection strategy for later tc_count calls on g. */
tc_status tc_set_strategy(tc_graph* g, int strategy);

/*
 * Planner settings of the count step (no counterpart in the paper; they
 * change speed, never results): params3[0] = work W(v) at or above which a
 * vertex may become CTA items, params3[1] = target wedges per CTA item (a
 * heavy vertex is split into chunks of about this size; each chunk stages
 * N_H(v) again), params3[2] = the same for warp items.  The next tc_count
 * re-plans.  Defaults 4096, a CTA chunk of the graph's wedges / (64 · SMs)
 * within [65536, 4194304] (set by the build), and 32768.
 */
tc_status tc_set_plan_params(tc_graph* g, const int64_t* params3);
tc_status tc_get_plan_params(const tc_graph* g, int64_t* out3);

/*
 * Optional device timing of every library kernel: when enabled, each
 * launch is bracketed by CUDA events on its own stream, and
 * tc_profile_read returns, per kernel name, the launch count and the
 * summed event time since the last reset.  The upload of host pairs in
 * tc_build_csr is timed too, as the entry "copy_h2d_pairs" (not a kernel:
 * tc_launch_count does not count it).  Timing adds two event records per
 * launch; leave it off for throughput runs.
 */
tc_status tc_profile_enable(int on);
tc_status tc_profile_reset(void);
/* Fills up to `cap` entries; returns the number of distinct kernels in *count. */
typedef struct { char name[48]; int64_t launches; double total_ms; } tc_kernel_time;
tc_status tc_profile_read(tc_kernel_time* out, int cap, int* count);

/* Number of kernels this library has launched since load (all threads). */
int64_t tc_launch_count(void);

/*
 * Testing aids for failure handling (no counterpart in the paper).
 * tc_debug_fail_allocation(k) arms one injected failure: the device
 * allocation the library requests k allocations from now (k = 0: the next
 * one) fails as if the device were out of memory; k < 0 disarms.  The
 * entry point that meets it frees what it had allocated and returns
 * TC_ERR_OUT_OF_MEMORY, and the next call works normally.  Process-wide
 * and shared by every thread (the server's workers included).
 * tc_debug_allocations counts the device allocations requested since the
 * library was loaded, tc_debug_live_allocations those currently held (by
 * graphs, batches and calls in flight).
 */
tc_status tc_debug_fail_allocation(int64_t k);
int64_t tc_debug_allocations(void);
int64_t tc_debug_live_allocations(void);

/*
 * Bounds-checked builds (compiled with -DTC_DEBUG_BOUNDS; the Python
 * binding's build(debug=True)): the count, gather and dense-core kernels
 * check every index they take from graph data against its array and, on a
 * failure, record it in an error word and skip to a valid entry instead of
 * faulting; each entry point then synchronises its stream and returns
 * TC_ERR_BOUNDS.  tc_debug_bounds_build returns 1 in such a build, else 0;
 * tc_debug_bounds_line the source line of the last failed check (0: none).
 */
int tc_debug_bounds_build(void);
int64_t tc_debug_bounds_line(void);

/* ------------------------------------------------------------------ batches
 * Many independent graphs processed as one: the batch is the disjoint union
 * of its graphs (graph k's vertices shifted by Σ_{j<k} n_j).  Triangles,
 * counts, flags and numerators of a disjoint union are those of each graph,
 * because Definition 1 only involves a vertex's neighbourhood; the only
 * per-graph quantity is the denominator 3△(G_k) = Σ_{v ∈ G_k} △(v).  One
 * build and one set of persistent count launches serve the whole batch.
 */
typedef struct tc_batch tc_batch;

/*
 * Builds a batch of num_graphs graphs.  Graph k has h_num_vertices[k]
 * vertices and the pairs [h_pair_offsets[k], h_pair_offsets[k+1]) of
 * src/dst, with ids local to the graph (in [0, n_k)).  h_pair_offsets
 * (num_graphs + 1 entries, first 0) and h_num_vertices are host arrays;
 * src/dst follow `flags` as in tc_build_csr.  Σ n_k must be < 2^31.
 * Errors as tc_build_csr (a local id outside its graph gives
 * TC_ERR_INVALID_ARG).  Synchronises `stream`.
 */
tc_status tc_batch_build(const void* src, const void* dst, const int64_t* h_pair_offsets,
                         const int64_t* h_num_vertices, int64_t num_graphs, uint32_t flags,
                         tc_stream stream, tc_batch** out);

/*
 * Counts and centrality of every graph of the batch.  Outputs are in union
 * labels (graph k's vertex i at index voff[k] + i; its canonical edges at
 * [eoff[k], eoff[k+1]) of the union edge list, see tc_batch_info); any may
 * be NULL:
 *   d_tri [Σn] uint64, d_edge_flag [Σm] uint8, d_numer [Σn] uint64,
 *   d_tc [Σn] double (NaN on the vertices of a triangle-free graph),
 *   d_tri_totals [num_graphs] uint64 = △(G_k).
 * Makes no host synchronisation and no allocation, so it may be captured
 * into a CUDA graph (after one plain run on the batch, which settles the
 * kernels' launch attributes).
 */
tc_status tc_batch_run(tc_batch* b, uint64_t* d_tri, uint8_t* d_edge_flag, uint64_t* d_numer,
                       double* d_tc, uint64_t* d_tri_totals, tc_stream stream);

/* Shape of a batch; the offset arrays (num_graphs + 1 entries each, host
 * memory, may be NULL) receive the vertex and canonical-edge offsets. */
tc_status tc_batch_info(const tc_batch* b, int64_t* num_graphs, int64_t* num_vertices,
                        int64_t* num_edges, int64_t* h_vertex_offsets, int64_t* h_edge_offsets);

/* The union's canonical edge list (union labels), as tc_copy_edges. */
tc_status tc_batch_copy_edges(const tc_batch* b, int32_t* d_u, int32_t* d_v, tc_stream stream);

tc_status tc_batch_get_stats(const tc_batch* b, tc_graph_stats* out);

/*
 * Autotuner: times the count step of this batch under several planner
 * settings (when a vertex is heavy enough for a CTA item; the work carried
 * by one CTA item and one warp item), `reps` runs each, keeps the fastest.
 * Synchronises `stream`.  tc_batch_get_params reports the chosen setting as
 * {cta_min_work, cta_chunk, warp_chunk}.
 */
tc_status tc_batch_autotune(tc_batch* b, int reps, tc_stream stream);
tc_status tc_batch_get_params(const tc_batch* b, int64_t* out3);

void tc_batch_free(tc_batch* b);

/*
 * Triangle counts, numerators and TC of a small graph given as a device
 * CSR, computed without allocating memory of any kind.  The paper has no
 * counterpart: this is a service for callers that cannot let a library
 * allocate — a runtime that owns all device memory through its own
 * allocator, a latency-critical loop that must not wait on pool growth, a
 * program whose memory footprint is fixed up front.  The results are those
 * of tc_count followed by tc_centrality on the same graph (Definition 1;
 * numerator and single division of Algorithm 2), bit for bit.
 *
 *   d_row_ptr  [n+1] int64, device: row v is d_col[d_row_ptr[v] ..
 *              d_row_ptr[v+1]); d_row_ptr[0] = 0, d_row_ptr[n] = nnz.
 *   d_col      [nnz] int32, device: neighbour ids in [0, n), each row
 *              strictly increasing (sorted, no duplicates), no self loops,
 *              symmetric (u in row v exactly when v in row u).
 *   n, nnz     0 <= n <= TC_NOALLOC_MAX_VERTICES, 0 <= nnz <=
 *              TC_NOALLOC_MAX_ENTRIES, nnz even (= 2m).
 *   d_tri      [n] uint64, device: △(v).  May be NULL.
 *   d_numer    [n] uint64, device: numer(v) = 3△(G)·TC(v).  May be NULL.
 *   d_tc       [n] double, device: TC(v); NaN everywhere if △(G) = 0.
 *              May be NULL.
 * Working memory is one fixed 768 KB array per device inside the library
 * (counts, edge flags, 3△(G), an error word); each call clears what it
 * uses first.  The first call on a device looks up that array's address
 * (with lazy module loading, it may also load the library's device code):
 * make that first call outside any stream capture.  Because the array is
 * shared, calls on the same device must not overlap: two calls in flight
 * at once, on different streams or threads, corrupt each other's results.
 * Order them on one stream, or with events.
 * Returns TC_ERR_INVALID_ARG, without touching the device, for sizes beyond
 * the limits, odd nnz or NULL inputs; TC_ERR_CUDA if the address lookup or
 * a launch fails; otherwise TC_OK once the work is enqueued on `stream`
 * (not synchronised; △(G) = 0 is not reported here).  An input that breaks
 * the CSR rules above (an id out of range, an unsorted or repeated row
 * entry, a self loop, an entry u in row v without v in row u, bad row
 * offsets) is detected on the device: every d_tri and d_numer entry is
 * then UINT64_MAX and every d_tc entry NaN.  d_tc alone cannot tell that
 * case from a triangle-free graph (NaN everywhere too): pass d_tri, which
 * is all zero for a valid triangle-free graph and all UINT64_MAX for a
 * rejected input.
 */
#define TC_NOALLOC_MAX_VERTICES 65536
#define TC_NOALLOC_MAX_ENTRIES 2097152
tc_status tc_csr_centrality_noalloc(const int64_t* d_row_ptr, const int32_t* d_col, int64_t n,
                                    int64_t nnz, uint64_t* d_tri, uint64_t* d_numer, double* d_tc,
                                    tc_stream stream);

/*
 * Serving: a request loop over the batch path (no counterpart in the
 * paper; it serves a stream of independent graphs).  Callers submit graphs
 * as host pair lists at any time; worker threads, each with its own
 * stream, take the waiting requests in arrival order and run as many of
 * them together as fit in one disjoint-union batch (up to max_batch_pairs
 * pairs and within the device-memory budget left by the batches in
 * flight), so requests that arrive while others run join the next batch.
 * With several workers, one batch's copies and build overlap another's
 * count and gather.  Each request gets exactly the results the same graph
 * gets alone (tc_count and tc_centrality on it).
 */
typedef struct tc_server tc_server;   /* opaque */

typedef struct {
    int64_t id;           /* as returned by tc_server_submit                  */
    int32_t status;       /* TC_OK, TC_NO_TRIANGLES or a negative tc_status   */
    int32_t batch_size;   /* requests in the batch that served this one       */
    uint64_t triangles;   /* △(G) of the request's graph                      */
    int64_t edges;        /* m: undirected edges after de-duplication         */
    double t_submit;      /* seconds since the server was created             */
    double t_start;       /* its batch began (copies, build, count, gather)   */
    double t_done;        /* its results were in the caller's buffers         */
} tc_request_info;

/*
 * Starts `workers` (1..8) worker threads on the current device.
 * memory_budget_bytes caps the device memory that running batches may
 * hold, by an estimate of each request's peak use; max_batch_pairs caps
 * the pairs of one batch (a larger single request still runs, alone).
 */
tc_status tc_server_create(int64_t memory_budget_bytes, int64_t max_batch_pairs, int workers,
                           tc_server** out);

/*
 * Queues one graph: num_pairs int32 pairs (h_src[i], h_dst[i]) in [0, n),
 * host memory (pinned memory moves fastest).  Results land in h_tri[n]
 * (△(v)) and h_tc[n] (TC(v)), host memory, either may be NULL.  All four
 * buffers must stay valid and untouched until the request is reported by
 * tc_server_poll.  Returns TC_ERR_OUT_OF_MEMORY at once, without touching
 * the device, when the request's own estimate exceeds the whole budget;
 * TC_ERR_STATE once the server is shutting down.  Never blocks on the GPU.
 */
tc_status tc_server_submit(tc_server* srv, const int32_t* h_src, const int32_t* h_dst,
                           int64_t num_pairs, int64_t n, uint64_t* h_tri, double* h_tc,
                           int64_t* request_id);

/*
 * Moves up to `cap` finished requests into out[], *count of them; waits up
 * to wait_ms milliseconds for the first one if none has finished.
 */
tc_status tc_server_poll(tc_server* srv, tc_request_info* out, int cap, int* count, int wait_ms);

/* Batches run so far, requests waiting, requests running, budget in use. */
tc_status tc_server_stats(tc_server* srv, int64_t* batches, int64_t* waiting, int64_t* running,
                          int64_t* memory_in_use);

/* Stops the server: batches already running finish (their result buffers
 * are filled), requests still waiting are dropped without running, then
 * the workers exit and the server is freed.  Poll until every request has
 * been reported first to receive all results. */
void tc_server_free(tc_server* srv);

/* Releases g.  Its device memory is freed in stream order on the stream of
 * the last call made on g, which must still exist. */
void tc_graph_free(tc_graph* g);
const char* tc_status_str(tc_status s);

#ifdef __cplusplus
}
#endif
#endif /* TC_GB300_H */
