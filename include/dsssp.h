/*
 * dsssp.h -- C ABI of the GB300 delta-stepping single-source shortest-path library.
 *
 * The method is the delta-stepping algorithm of Meyer and Sanders as restated
 * in linear-algebra form by Sridhar et al., "Delta-stepping SSSP: from Vertices
 * and Edges to GraphBLAS Implementations" (IPDPSW 2019):
 *   - Section III-A / Fig. 1: split every vertex's out-arcs into light
 *     (weight <= Delta) and heavy (weight > Delta) sets, A_L and A_H;
 *   - Section III-B: bucket B_i holds the vertices with i*Delta <= t < (i+1)*Delta;
 *   - Section IV-C / Fig. 1 (left): the light relaxation of bucket i is the masked
 *     min-plus product t_Req = A_L^T (t o t_Bi), repeated until no vertex
 *     re-enters B_i; then one heavy pass t_Req = A_H^T (t o S) over the set S of
 *     vertices processed in the bucket; then the next non-empty bucket.
 *
 * Conventions shared by every entry point:
 *   - A graph is directed; CSR row v lists the out-arcs of v (Section II-A).
 *     row_ptr has n+1 int64 entries, col has m int32 heads, weights are m int32
 *     or m float32 values. Self-loops and repeated arcs are accepted.
 *   - Weights must be non-negative and finite (NaN, +-inf and negative values
 *     are rejected). A float32 -0.0 is stored as +0.0.
 *   - Path sums use the weight type's own addition: float32 adds round to
 *     nearest-even after every arc; int32 adds are exact. Distances are the
 *     least fixed point of d[s] = 0, d[v] = min_(u,v) d[u] (+) w; every
 *     relaxation order reaches the same bits.
 *   - Overflow (the paper assumes exact reals, Section III; this library's own
 *     boundary): when some arc (u,v) out of a reached u has a sum d[u] (+) w(u,v)
 *     that the weight type cannot hold -- an int32 sum >= INT32_MAX (the value
 *     that marks "unreachable"), or a float32 sum that rounds to +inf -- the solve
 *     returns DSSSP_ERR_OVERFLOW and writes no output. The condition is taken on
 *     the final distances, so it does not depend on the relaxation order.
 *   - pred[v] is the smallest u with an arc (u,v) such that d[u] (+) w(u,v) == d[v];
 *     pred[src] = src; unreached vertices get dist = +inf (float32) or
 *     INT32_MAX (int32) and pred = -1.
 *   - Every pointer to vertex or arc data is a DEVICE pointer of the current
 *     CUDA device unless the argument says otherwise. `stream` is a
 *     cudaStream_t passed as void*; NULL means the legacy default stream.
 *     All device work is ordered on that stream.
 *   - Functions return a dsssp_status and never abort the process. Device-side
 *     failures (a timed-out wait, a phase cap) are reported as status codes,
 *     never as a trap.
 *   - Limits: 1 <= n <= 2^31 - 2 and m <= 2^31 - 1.
 */
#ifndef DSSSP_H
#define DSSSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DSSSP_OK = 0,
    DSSSP_ERR_INVALID_ARG = 1,   /* a scalar argument is out of range or a pointer is NULL      */
    DSSSP_ERR_BAD_GRAPH = 2,     /* row_ptr not monotone / not starting at 0, head out of range  */
    DSSSP_ERR_NEG_WEIGHT = 3,    /* a weight is negative, NaN or infinite                        */
    DSSSP_ERR_NOT_CONVERGED = 4, /* the phase cap of dsssp_options.max_phases was reached       */
    DSSSP_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out (dsssp_options.timeout_ns) */
    DSSSP_ERR_CUDA = 6,          /* a CUDA runtime call failed                                   */
    DSSSP_ERR_NO_TAPE = 7,       /* dsssp_backward on a batch without a recorded tree            */
    DSSSP_ERR_OOM = 8,           /* a device allocation failed                                   */
    DSSSP_ERR_UNSUPPORTED = 9,   /* the device or launch shape cannot run this entry point      */
    DSSSP_ERR_TOO_LARGE = 10,    /* the graph exceeds dsssp_solve_noalloc's fixed working memory */
    DSSSP_ERR_DEGENERATE = 11,   /* the predecessor graph has a cycle (zero-weight ties): no gradient */
    DSSSP_ERR_OVERFLOW = 12      /* a path sum out of a reached vertex does not fit the weight type */
} dsssp_status;

typedef enum { DSSSP_I32 = 0, DSSSP_F32 = 1 } dsssp_dtype;

/* Opaque graph handle: a device copy of the CSR plus the per-Delta light/heavy
 * layouts and the solver workspace. Owned by the library. */
typedef struct dsssp_graph dsssp_graph;

/* Solver execution schemes (dsssp_options.mode). */
typedef enum {
    DSSSP_MODE_PERSISTENT = 0,   /* one cooperative kernel runs every phase; grid-wide barriers  */
    DSSSP_MODE_STEPPED = 1,      /* one kernel launch per phase, loop driven by the host          */
    DSSSP_MODE_DENSE = 2,        /* the paper's full-vector form (Fig. 1 left; the filter fusion of
                                    Section VI-B): t_Bi, S and the far pile are per-vertex stamps,
                                    every phase scans all n of them and filters each scanned row
                                    into light or heavy arcs on the fly. Same results; block_size,
                                    grid_size, solo_work, flags other than ASYNC and test_hook are
                                    ignored; stats fill buckets, light_phases and heavy_phases. */
    DSSSP_MODE_TEAM = 3          /* the solve as one instance of the batch kernel on a single
                                    thread-block cluster of dsssp_options.team_blocks blocks (0: 16, or 8
                                    where 16 cannot be scheduled): phases end in a hardware cluster
                                    barrier and the control stays in shared memory, which suits graphs
                                    with many small phases (high diameter, small frontiers). Same
                                    results; block_size, grid_size, solo_work, timeout_ns and test_hook
                                    are ignored; stats fill the phase, arc and vertex counters,
                                    rebin_phases = next-bucket selections, ns_total, grid_size = blocks */
} dsssp_mode;

/* dsssp_options.flags */
#define DSSSP_FLAG_ASYNC 0x1u    /* do not wait for the solve: device-side status is kept in the
                                    graph and returned by dsssp_graph_sync()                        */
#define DSSSP_FLAG_NO_FUSE 0x2u  /* keep every heavy pass in a phase of its own; by default, when
                                    bucket i+1 already holds vertices, bucket i's heavy pass and
                                    bucket i+1's first light round share one phase (same results)   */

/* Test hooks (dsssp_options.test_hook): exercise error paths without a fault. */
#define DSSSP_HOOK_NONE 0
#define DSSSP_HOOK_STALL_BARRIER 1  /* block 1 leaves the persistent kernel before its first
                                       barrier, so the others' bounded wait runs out and the
                                       solve returns DSSSP_ERR_TIMEOUT                           */

typedef struct {
    uint32_t struct_size;   /* sizeof(dsssp_options); 0 fields mean "default"                  */
    uint32_t flags;         /* DSSSP_FLAG_*                                                      */
    int32_t  mode;          /* dsssp_mode; default DSSSP_MODE_PERSISTENT                        */
    int32_t  block_size;    /* threads per block, multiple of 32, <= 512; default 512           */
    int32_t  grid_size;     /* blocks of the persistent kernel; default = all co-resident blocks */
    int32_t  solo_work;     /* phases with at most this many arcs or list entries run on one
                               block without grid barriers; default 2048, -1 disables            */
    int64_t  max_phases;    /* cap on phases (barrier steps); default 2^26                       */
    int64_t  timeout_ns;    /* limit of any single device-side wait; default 2e9 (2 s)           */
    int32_t  test_hook;     /* DSSSP_HOOK_*                                                      */
    int32_t  team_blocks;   /* batches and DSSSP_MODE_TEAM solves: blocks per instance (a
                               thread-block cluster of 1, 2, 4, 8 or 16; 16 is a non-portable
                               cluster size, UNSUPPORTED where it cannot be co-scheduled);
                               0 = automatic (batches: 1-8, more blocks per instance when
                               instances are few; team solves: 16, else 8). Batches only: -1 =
                               the instances one after another, each by the grid-wide persistent
                               solver (no tape; a run then cannot be captured into a CUDA graph) */
    int32_t  reserved[4];
} dsssp_options;

/* Counters of one solve (filled when a non-NULL pointer is passed; this makes
 * the call wait for the solve). Times are device-side (%globaltimer), per phase kind. */
typedef struct {
    int64_t buckets;          /* non-empty buckets processed                                   */
    int64_t light_phases;     /* light relaxation rounds (inner loop of Fig. 1)                */
    int64_t heavy_phases;     /* heavy passes                                                   */
    int64_t rebin_phases;     /* refills of the bucket-slot window from the overflow list       */
    int64_t vertices_light;   /* sum of |frontier| over light rounds                           */
    int64_t vertices_heavy;   /* sum of |S| over heavy passes                                   */
    int64_t arcs_light;       /* light arcs relaxed                                             */
    int64_t arcs_heavy;       /* heavy arcs relaxed                                             */
    int64_t far_scanned;      /* overflow entries examined by window refills                    */
    int64_t improvements;     /* strict distance decreases                                      */
    int64_t ns_light;         /* device time in light rounds                                    */
    int64_t ns_heavy;         /* device time in heavy passes                                    */
    int64_t ns_rebin;         /* device time in window refills                                  */
    int64_t ns_total;         /* device time of the whole solve kernel                          */
    int64_t ns_first_arrival; /* sum over phases: phase start to the first block's barrier arrival */
    int64_t ns_arrival_spread;/* sum over phases: first to last barrier arrival                  */
    int64_t grid_size;        /* blocks used                                                    */
    int64_t block_size;       /* threads per block used                                          */
    int64_t reserved[6];
} dsssp_stats;

/* Human-readable name of a status code (static string, never NULL). */
const char *dsssp_status_string(dsssp_status s);

/* Fill *opt with the defaults above. */
dsssp_status dsssp_options_default(dsssp_options *opt);

/* Create a graph handle: validates and copies the CSR to the current device.
 * Section II-A (adjacency matrix, row = out-arcs), Section III-A (weights).
 *   n, m        vertex and arc counts (limits in the file header);
 *   row_ptr     int64[n+1], col int32[m], w int32[m] or float32[m];
 *   dtype       DSSSP_I32 or DSSSP_F32;
 *   device_ptrs 1: row_ptr/col/w are device pointers; 0: host pointers;
 *   stream      ordering stream for the copies and validation;
 *   out         receives the handle (owned by the library until dsssp_graph_destroy).
 * The caller's buffers are not retained. Waits for validation to finish.
 * Errors: INVALID_ARG, BAD_GRAPH, NEG_WEIGHT, OOM, CUDA. */
dsssp_status dsssp_graph_create(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                const void *w, dsssp_dtype dtype, int device_ptrs, void *stream,
                                dsssp_graph **out);

/* Release a handle and all device memory it owns (waits for its pending work). */
dsssp_status dsssp_graph_destroy(dsssp_graph *g);

/* Query a handle: any output pointer may be NULL. */
dsssp_status dsssp_graph_info(const dsssp_graph *g, int64_t *n, int64_t *m, int32_t *dtype);

/* Light/heavy split for one Delta (Section III-A, Section IV-A, Fig. 1:
 * A_L = A o (A <= Delta), A_H = A o (A > Delta)). Builds, on `stream`, a copy
 * of the arcs in which every row lists its light arcs first, then its heavy
 * arcs, each group in input order; caches it in the handle (a few Deltas are
 * kept, least recently used evicted). dsssp_solve calls this itself when
 * needed; calling it first lets the split be timed on its own.
 * delta > 0, may be +inf (every arc light). Errors: INVALID_ARG, OOM, CUDA. */
dsssp_status dsssp_prepare(dsssp_graph *g, double delta, void *stream);

/* One delta-stepping solve (Fig. 1; Section III-C, IV-C, IV-D):
 *   src    source vertex, 0 <= src < n;
 *   delta  bucket width, > 0 (may be +inf);
 *   dist   device int32[n] or float32[n] (the graph's dtype), written on success;
 *   pred   device int32[n], written on success (may be NULL);
 *   opt    NULL for defaults;
 *   stats  NULL, or host struct filled after the solve (then the call waits);
 * Unless DSSSP_FLAG_ASYNC is set the call waits for the solve and returns its
 * device-side status. Solves on one handle share its workspace: issue them on
 * one stream (or serialize them). Errors: INVALID_ARG, TIMEOUT, NOT_CONVERGED,
 * OVERFLOW, OOM, CUDA, UNSUPPORTED. */
dsssp_status dsssp_solve(dsssp_graph *g, int32_t src, double delta, void *dist, int32_t *pred,
                         const dsssp_options *opt, dsssp_stats *stats, void *stream);

/* Wait for the handle's outstanding work on `stream` and return (and clear)
 * the first device-side status recorded by asynchronous solves. */
dsssp_status dsssp_graph_sync(dsssp_graph *g, void *stream);

/* A solve that allocates no memory at all. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code that runs
 * under an allocator it must not bypass, within a memory budget fixed in
 * advance, or where a device allocation would synchronise the device or fail.
 * It returns the same distances and predecessors as dsssp_solve (bit for bit),
 * reading the caller's CSR directly and keeping all of its working state in one
 * fixed array compiled into the library (about 11 MB, held by every GPU that
 * loads the library until the process exits).
 *   n           number of vertices, 1 <= n <= 131072 (larger graphs:
 *               DSSSP_ERR_TOO_LARGE); m arcs, m <= 2^31 - 1;
 *   row_ptr, col, w   DEVICE pointers: int64[n+1], int32[m], int32 or float32[m]
 *               (dtype); read only, never copied or modified;
 *   src, delta  as for dsssp_solve;
 *   dist, pred  DEVICE outputs, n entries each (pred may be NULL), written only
 *               on success.
 * The call validates the CSR on the device and waits for the solve (it reads
 * the result status back to the host), so it cannot run while `stream` is being
 * captured into a CUDA graph: it then returns DSSSP_ERR_UNSUPPORTED without
 * touching the stream. The first call on a device looks up the device address
 * of the fixed array (once per device, with that device current). Every call
 * uses the same array and clears what it needs first, so calls that overlap on
 * the GPU (for example on two streams) race: serialise them. A barrier wait
 * gives up after 2 s without progress (no block arrived and no long row
 * advanced) and returns DSSSP_ERR_TIMEOUT.
 * Errors: INVALID_ARG, TOO_LARGE, BAD_GRAPH, NEG_WEIGHT, TIMEOUT, NOT_CONVERGED,
 * OVERFLOW, CUDA, UNSUPPORTED. */
dsssp_status dsssp_solve_noalloc(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                 const void *w, dsssp_dtype dtype, int32_t src, double delta,
                                 void *dist, int32_t *pred, void *stream);

/* ------------------------------------------------------------------------ */
/* Batches: many independent solves in one persistent launch.               */
/*                                                                          */
/* Delta-stepping's parallelism within one solve is the work of one bucket   */
/* phase (Section III-C); independent solves -- many sources on one graph,   */
/* or many graphs -- add a second, coarser dimension. A batch solves every   */
/* instance with the same method and the same exact results as dsssp_solve;  */
/* each instance keeps its own bucket state and is processed start to end by */
/* one team -- a block, or a thread-block cluster of up to 8 blocks -- of a  */
/* persistent kernel whose teams take instances from a device-side           */
/* queue (largest graphs first). A batch is a plan: its instance table,      */
/* working memory and a CUDA graph of its launch are built once, then run    */
/* any number of times.                                                     */

typedef struct dsssp_batch dsssp_batch;

/* dsssp_batch_create flags */
#define DSSSP_BATCH_TAPE 0x1u    /* record every instance's shortest-path tree (parent and the input
                                    index of its tree arc) for dsssp_backward; float32 graphs only */

/* dsssp_backward flags */
#define DSSSP_BACKWARD_ACCUMULATE 0x1u  /* add into grad_w instead of overwriting it            */

/* Counters of one instance of the last run (dsssp_batch_sync). */
typedef struct {
    int64_t buckets;          /* non-empty buckets processed                                   */
    int64_t light_phases;     /* light relaxation rounds                                        */
    int64_t heavy_phases;     /* heavy passes                                                   */
    int64_t select_phases;    /* next-bucket selections (scans of the instance's far list)      */
    int64_t arcs_light;       /* light arcs relaxed                                             */
    int64_t arcs_heavy;       /* heavy arcs relaxed                                             */
    int64_t improvements;     /* strict distance decreases                                      */
    int64_t far_scanned;      /* far-list entries examined by selections                        */
    int64_t ns;               /* device time from the instance's start to its end              */
    int64_t team;             /* block that solved it                                           */
    int64_t vertices_light;   /* sum of |frontier| over light rounds                           */
    int64_t vertices_heavy;   /* sum of |S| over heavy passes                                   */
    int64_t reserved[4];
} dsssp_batch_stats;

/* Build a batch (a plan of n_inst solves):
 *   graphs      HOST array of n_graphs handles, all of one dtype and on the current device;
 *   delta       HOST array of n_graphs bucket widths (> 0, may be +inf), one per graph;
 *   n_inst      number of solves, >= 1;
 *   src         HOST array of n_inst sources (0 <= src < n of its graph);
 *   src_graph   HOST array of n_inst graph indices, or NULL: every instance on graphs[0];
 *   dist        HOST array of n_inst DEVICE pointers, each n (of its graph) elements of the
 *               graph's dtype, written by every run;
 *   pred        HOST array of n_inst DEVICE pointers (int32[n]) or NULL entries, or NULL;
 *   flags       DSSSP_BATCH_TAPE or 0;
 *   opt         NULL, or options (block_size must be 512 or 0; grid_size caps the number of
 *               blocks; max_phases caps the phases of each instance; team_blocks sets how many
 *               blocks -- a thread-block cluster sharing the instance's control through
 *               distributed shared memory -- solve one instance: 1, 2, 4, 8, 16, or 0 for automatic);
 *   stream      orders the set-up work (light/heavy splits, tables); the call waits for it;
 *   out         receives the plan.
 * The plan keeps the graphs' splits for these Deltas alive (a graph holds at most four) and
 * the output pointers; graphs must outlive the plan. The caller's arrays are not retained.
 * Errors: INVALID_ARG, UNSUPPORTED (int32 graphs with DSSSP_BATCH_TAPE, more than four
 * Deltas held on one graph), OOM, CUDA. */
dsssp_status dsssp_batch_create(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta,
                                int32_t n_inst, const int32_t *src, const int32_t *src_graph,
                                void *const *dist, int32_t *const *pred, uint32_t flags,
                                const dsssp_options *opt, void *stream, dsssp_batch **out);

/* Enqueue one run of every instance on `stream`: a single launch of the plan's CUDA graph
 * (queue reset + the persistent kernel). While `stream` is being captured into a caller's CUDA
 * graph, the two operations are enqueued directly and become nodes of that graph. Allocates
 * nothing and does not wait. A plan with team_blocks = -1 enqueues one dsssp_solve per instance
 * instead (the first run may allocate the graphs' workspaces; UNSUPPORTED while capturing).
 * Errors: INVALID_ARG, CUDA, UNSUPPORTED. */
dsssp_status dsssp_batch_run(dsssp_batch *b, void *stream);

/* Wait for `stream`, then return (and clear) the first device-side status of the runs and
 * backward passes since the last sync (NOT_CONVERGED when an instance hit the phase cap,
 * OVERFLOW when a path sum of an instance overflowed -- in both cases that instance's outputs
 * are not written -- and DEGENERATE from dsssp_backward). stats: NULL or a HOST array of n_inst records, filled
 * from the last run, in the caller's instance order. */
dsssp_status dsssp_batch_sync(dsssp_batch *b, dsssp_batch_stats *stats, void *stream);

/* Release a plan (waits for its pending work). */
dsssp_status dsssp_batch_destroy(dsssp_batch *b);

/* Convenience: create, run once, sync (stats as above, may be NULL), destroy. */
dsssp_status dsssp_solve_batched(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta,
                                 int32_t n_inst, const int32_t *src, const int32_t *src_graph,
                                 void *const *dist, int32_t *const *pred, const dsssp_options *opt,
                                 dsssp_batch_stats *stats, void *stream);

/* Adjoint of the distances with respect to the weights. The paper has no counterpart: it is
 * the gradient of L = sum over instances k and reached vertices v of c_k[v] * dist_k[v] for
 * the distances of the last run of a batch created with DSSSP_BATCH_TAPE. Within the
 * shortest-path tree of instance k, dist_k[v] is the sum of the weights on the tree path
 * from the source to v, so dL/dw(u,v) = sum of c_k[x] over the subtree below v when (u,v) is
 * v's tree arc, and 0 for arcs outside every tree. The tree is taken from the forward run
 * (the input arc that realised dist[v] -- among all arcs whose sum reaches dist[v], the one
 * with the smallest input index, whose tail is pred[v]); nothing is re-solved. At such a tie
 * L has a kink and this rule picks one subgradient. Subtree sums are accumulated
 * leaves first in float64 and rounded to float32 once.
 *   c       HOST array of n_inst DEVICE pointers, float32[n] each (entries of unreached
 *           vertices are ignored);
 *   grad_w  HOST array of n_graphs DEVICE pointers, float32[m] each, indexed like the
 *           weights given to dsssp_graph_create;
 *   flags   DSSSP_BACKWARD_ACCUMULATE or 0.
 * Ordered on `stream`; does not wait. Errors: INVALID_ARG, NO_TAPE (no tape, or no run yet),
 * CUDA; DEGENERATE (the predecessor graph of some instance has a cycle) is reported by the
 * next dsssp_batch_sync. */
dsssp_status dsssp_backward(dsssp_batch *b, const float *const *c, float *const *grad_w, uint32_t flags,
                            void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuning of Delta. The paper fixes Delta by hand (Section VI-A uses      */
/* Delta = 1 on unit weights); delta-stepping's work and phase count trade    */
/* off through Delta (Section III: small Delta approaches Dijkstra's order,  */
/* large Delta Bellman-Ford's). The tuner times sample solves on this GPU    */
/* and returns, per graph, the Delta with the least device time.             */

/* dsssp_tune_options.target */
#define DSSSP_TUNE_SOLVE 0   /* time dsssp_solve, one sample source after another                 */
#define DSSSP_TUNE_BATCH 1   /* time instances of a batch (each on one block, as dsssp_batch_run)  */

typedef struct {
    uint32_t struct_size;    /* sizeof(dsssp_tune_options)                                        */
    int32_t  target;         /* DSSSP_TUNE_SOLVE or DSSSP_TUNE_BATCH                              */
    int32_t  n_candidates;   /* 0: a ladder of 7 powers of two around mean weight / mean degree x 4  */
    int32_t  refine;         /* refinement rounds (each tries the best x 2^(+-1/2^r)); default 2, -1: none */
    double   candidates[16]; /* explicit candidates (> 0) when n_candidates > 0                   */
    int32_t  reserved[8];
} dsssp_tune_options;

/* Choose Delta for every graph:
 *   graphs       HOST array of n_graphs handles (one dtype, current device);
 *   sample_src   HOST array of n_graphs * k sample sources (k per graph, graph-major);
 *   opt          NULL for defaults (DSSSP_TUNE_SOLVE, default ladder, 2 refinement rounds);
 *   delta_out    HOST array of n_graphs: the chosen Delta;
 *   ms_out       NULL or HOST array of n_graphs: device time of the k samples at that Delta.
 * With DSSSP_TUNE_BATCH every (graph, candidate, source) is one instance of a tuning batch
 * and its cost is that instance's device time. The light/heavy splits the tuner builds stay
 * cached in the handles. Waits for its work. Errors: INVALID_ARG, OOM, CUDA and those of
 * dsssp_solve / dsssp_batch_create. */
dsssp_status dsssp_autotune(dsssp_graph *const *graphs, int32_t n_graphs, const int32_t *sample_src, int32_t k,
                            const dsssp_tune_options *opt, double *delta_out, double *ms_out, void *stream);

/* Choose dsssp_options.solo_work for single solves of one graph at one Delta: times k sample
 * solves with the solo threshold at -1 (off), 512, 2048, 8192 and 32768 arcs and returns the
 * fastest in solo_work_out (ms_out, may be NULL: their device time). Waits for its work.
 * Errors: INVALID_ARG and those of dsssp_solve. */
dsssp_status dsssp_tune_solo_work(dsssp_graph *g, const int32_t *sample_src, int32_t k, double delta,
                                  int32_t *solo_work_out, double *ms_out, void *stream);

/* Choose the scheme of single solves of one graph at one Delta: times k sample solves in the
 * persistent mode at the solo thresholds of dsssp_tune_solo_work and in DSSSP_MODE_TEAM with 8 and
 * 16 blocks (a size that cannot be scheduled here is skipped), and writes to *opt_out the default
 * options with the fastest scheme's mode, solo_work and team_blocks; ms_out (may be NULL) receives
 * its device time. The paper fixes no schedule (Section VI); delta-stepping phases are small on
 * high-diameter graphs and large on small-world ones, which favours one scheme or the other.
 * Waits for its work. Errors: INVALID_ARG and those of dsssp_solve. */
dsssp_status dsssp_tune_schedule(dsssp_graph *g, const int32_t *sample_src, int32_t k, double delta,
                                 dsssp_options *opt_out, double *ms_out, void *stream);

/* Choose the team size of a batch (dsssp_options.team_blocks: blocks per instance, 1, 2, 4, 8
 * or 16, and -1 -- one instance after another on the whole GPU -- when every instance is on one
 * graph; sizes that cannot be co-scheduled are skipped) by timing the whole batch at each size: builds the plan the arguments describe (as
 * dsssp_batch_create, outputs written) once per size, runs it twice and keeps the fastest
 * second run. team_blocks_out receives the size; ms_out (may be NULL) its device time.
 * Waits for its work. Errors: those of dsssp_batch_create / run / sync. */
dsssp_status dsssp_tune_team_blocks(dsssp_graph *const *graphs, int32_t n_graphs, const double *delta,
                                    int32_t n_inst, const int32_t *src, const int32_t *src_graph,
                                    void *const *dist, int32_t *const *pred, int32_t *team_blocks_out,
                                    double *ms_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DSSSP_H */
