/*
 * fg -- fixpoint graph relaxation on NVIDIA GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of the Falcon method (Gogoi,
 * Cheramangalath and Nasre, "Custom Code Generation for a Graph DSL",
 * arXiv 1903.01665): the edge-relaxation sweep repeated until a fixpoint for
 * single-source shortest paths (Alg. 1 and 2), breadth-first search (Alg. 3)
 * and connected components (benchmarked in Sec. 4), in the four variants the
 * paper generates from one specification (Sec. 3.1-3.3):
 *
 *   FG_VERTEX_SYNC  vertex-based over CSR (points x outnbrs, Alg. 1),
 *                   double-buffered values, one grid barrier per round;
 *   FG_EDGE_SYNC    edge-based over the COO edge list (edges, Alg. 2),
 *                   double-buffered values, one grid barrier per round;
 *   FG_VERTEX_ASYNC data-driven (Sec. 3.3): a device worklist of vertices,
 *                   in-place atomic MIN, run until the worklist is empty; an
 *                   SSSP generation whose worklist holds a quarter of the
 *                   vertices with out-edges or more tests every vertex
 *                   instead (queued, or lowered during the generation);
 *   FG_EDGE_ASYNC   the same worklist expanded to its out-edges and relaxed
 *                   edge-parallel, in place; a generation whose worklist holds
 *                   a quarter of the edges or more (BFS: half) streams the
 *                   whole edge list instead, relaxing the edges whose source
 *                   is queued;
 *
 * and a fifth built on the paper's in-neighbour iterator (innbrs, Sec. 2):
 *
 *   FG_PULL         vertex-based, double-buffered, direction-optimising: a
 *                   round in which many vertices changed pulls over the
 *                   in-neighbours (SSSP/CC: each vertex takes the minimum of
 *                   its in-neighbours' candidates, no atomics; BFS bottom-up:
 *                   an unvisited vertex stops at its first in-neighbour on
 *                   the frontier), the other rounds push as FG_VERTEX_SYNC.
 *                   The transposed CSR it reads is built on the first pull
 *                   query of a graph and kept with it (about 8 bytes per edge);
 *
 * and a sixth for high-diameter graphs:
 *
 *   FG_BUCKET       FG_VERTEX_ASYNC with the worklist split by distance
 *                   (near-far, a two-bucket form of delta-stepping): SSSP
 *                   vertices whose new distance is below a threshold T are
 *                   processed first; the others wait in a far list, and when
 *                   the near worklist runs empty T moves to the far list's
 *                   smallest distance + delta and the far list is split.
 *                   BFS and CC run as FG_VERTEX_ASYNC.
 *
 * All reach the same unique fixpoint, so their outputs are identical.
 *
 * Conventions for every call:
 *   - Ids, weights, distances, levels and labels are int32.  "Unreached" is
 *     INT32_MAX (FG_INF) for SSSP and BFS.
 *   - Input and output arrays may be host memory (pageable or pinned) or
 *     device memory of the current device; the library tells them apart
 *     with cudaPointerGetAttributes.  Inputs are read during the call only
 *     and never retained.  Outputs are caller-owned int32[n], written once,
 *     in bulk, only on success (one transfer per attribute array, as the
 *     paper's data-transfer aggregation prescribes for attributes read back
 *     on the host).
 *   - Every call returns an fg_status; nothing throws across the ABI.  On
 *     error, fg_last_error() gives a message for the calling thread and the
 *     outputs are untouched.
 *   - A graph handle is immutable after creation (a FG_GRAPH_LAZY graph
 *     only adds the parts it builds on first use, under a lock) and may be
 *     queried from several host threads and streams at once; each query
 *     owns its state.
 *   - Queries run on the calling thread's current CUDA device, which must
 *     be the device the graph was created on.
 */
#ifndef FG_H
#define FG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FG_INF 2147483647

typedef struct fg_graph fg_graph;

typedef enum {
    FG_OK = 0,
    FG_ERR_INVALID_ARG = 1,     /* null pointer, n <= 0, m < 0, id outside [0,n), bad
                                   row offsets, invalid mode/algo, wrong device */
    FG_ERR_NEGATIVE_WEIGHT = 2, /* some weight < 0 (create time) */
    FG_ERR_OVERFLOW = 3,        /* a finite shortest distance is >= INT32_MAX */
    FG_ERR_OUT_OF_MEMORY = 4,   /* device or host allocation failed */
    FG_ERR_TIMEOUT = 5,         /* round cap reached, or a device-side wait ran out */
    FG_ERR_CUDA = 6             /* any other CUDA runtime error */
} fg_status;

typedef enum {
    FG_VERTEX_SYNC = 0,
    FG_VERTEX_ASYNC = 1,
    FG_EDGE_SYNC = 2,
    FG_EDGE_ASYNC = 3,
    FG_AUTO = 4,                /* the mode fg_select_mode picks */
    FG_PULL = 5,
    FG_BUCKET = 6
} fg_mode;

typedef enum { FG_ALGO_SSSP = 0, FG_ALGO_BFS = 1, FG_ALGO_CC = 2 } fg_algo;

/*
 * Graph creation.
 *
 * fg_graph_create_csr: n vertices, m edges in compressed sparse rows (the
 *   storage of vertex-based code, Sec. 3.1): row_off[n+1] int64, row_off[0]
 *   = 0, non-decreasing, row_off[n] = m; col[m] int32 targets in [0,n);
 *   w[m] int32 weights >= 0, or NULL for all-ones weights.
 * fg_graph_create_coo: the same graph as an edge list (source, destination,
 *   weight) in any order (the storage of edge-based code, Sec. 3.1).
 *
 * Both build, on the device: the CSR (uint32 offsets; m < 2^32 required),
 * the source-sorted COO (its dst and w arrays are the CSR's col and w), the
 * degree buckets of the vertex kernels (1..31, 32..1023, >= 1024 out-edges),
 * and the symmetrised CSR/COO used by connected components (every edge also
 * read backwards: the undirected nbrs iterator, Table "foreach iterators").
 * Self-loops and duplicate edges are kept.  The handle is written to *out
 * only on success.  Errors: FG_ERR_INVALID_ARG, FG_ERR_NEGATIVE_WEIGHT,
 * FG_ERR_OUT_OF_MEMORY, FG_ERR_CUDA.
 */
fg_status fg_graph_create_csr(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                              const int32_t *w, fg_graph **out);
fg_status fg_graph_create_coo(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                              const int32_t *w, fg_graph **out);

/*
 * The same with creation flags (0 = the plain calls above).
 *
 * FG_GRAPH_LAZY   keep only the CSR and its degree buckets at creation (R-MAT
 *                 22: 0.6 GB of the 1.95 GB a full build holds).  The COO's
 *                 source array is built by the first edge-based query on the
 *                 directed graph (FG_EDGE_SYNC, FG_EDGE_ASYNC, fg_sweep's
 *                 edge variant, the transposed view of FG_PULL, or an SSSP
 *                 whose overflow check runs), the symmetrised view by the
 *                 first CC query; each is kept with the graph.  The call
 *                 that builds a part also pays for it, and an out-of-memory
 *                 error can then come from a query; fg_graph_info reports
 *                 device_bytes as it grows and n_isolated as -1 until the
 *                 symmetrised view exists.  Results are identical.
 * FG_GRAPH_RELABEL  renumber the vertices internally, by in-degree class
 *                 (floor(log2(in-degree)), highest first; original order
 *                 within a class), so that the most probed targets share
 *                 cache lines and stay in L2.  Every call still takes and
 *                 returns original ids: a query's source is translated on
 *                 the device, its output permuted back, and CC labels stay
 *                 the minimum original id of each component.  Costs 8
 *                 bytes per vertex and, per query, one gather of the output
 *                 (CC: two passes).
 * FG_GRAPH_KEEP_IDS  never renumber.
 * Neither flag: renumber when the in-degrees are skewed (their Gini
 *                 coefficient above 0.5: R-MAT yes, grids no).
 *                 fg_graph_info's relabelled field tells which.
 *
 * Unknown flag bits, or both FG_GRAPH_RELABEL and FG_GRAPH_KEEP_IDS:
 * FG_ERR_INVALID_ARG.
 */
#define FG_GRAPH_LAZY 1u
#define FG_GRAPH_RELABEL 2u
#define FG_GRAPH_KEEP_IDS 4u
fg_status fg_graph_create_csr_ex(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                                 const int32_t *w, uint32_t flags, fg_graph **out);
fg_status fg_graph_create_coo_ex(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 const int32_t *w, uint32_t flags, fg_graph **out);

/* Frees the graph's device memory.  NULL is accepted (no-op). */
fg_status fg_graph_destroy(fg_graph *g);

/* Host-side facts about a graph, computed at creation (device_bytes and
   n_isolated also when a FG_GRAPH_LAZY graph builds a part). */
typedef struct {
    int32_t n;
    int64_t m;
    int64_t m_sym;              /* edges of the symmetrised graph (2m) */
    int32_t max_out_degree;
    int32_t n_zero_out;         /* vertices with no out-edge */
    int32_t n_low, n_mid, n_high; /* degree-bucket sizes (1..31, 32..1023, >= 1024) */
    int32_t n_high_chunks;      /* 2048-edge chunks of the high bucket */
    int32_t n_isolated;         /* vertices with no edge in either direction (-1 until a
                                   FG_GRAPH_LAZY graph has built its symmetrised view) */
    int64_t device_bytes;       /* device memory held by the handle */
    int32_t relabelled;         /* 1 if the vertices are renumbered internally
                                   (FG_GRAPH_RELABEL, or skewed in-degrees) */
    float in_degree_gini;       /* Gini coefficient of the in-degrees (binned) */
} fg_graph_info_t;

fg_status fg_graph_info(const fg_graph *g, fg_graph_info_t *out);

/*
 * Queries.  src in [0,n).  out is int32[n]:
 *   fg_sssp: shortest distance from src (Alg. 1/2 fixpoint), FG_INF if
 *            unreachable.  FG_ERR_OVERFLOW if a finite distance would be
 *            >= INT32_MAX.
 *   fg_bfs:  fewest edges on a path from src (Alg. 3 fixpoint), FG_INF if
 *            unreachable; weights are ignored.
 *   fg_cc:   smallest vertex id of the vertex's component in the symmetrised
 *            graph (weak components of the directed input).
 * The call blocks until out is written.  Uses the legacy default stream.
 */
fg_status fg_sssp(const fg_graph *g, int32_t src, int32_t *dist_out, fg_mode mode);
fg_status fg_bfs(const fg_graph *g, int32_t src, int32_t *level_out, fg_mode mode);
fg_status fg_cc(const fg_graph *g, int32_t *label_out, fg_mode mode);

/*
 * The runtime form of the paper's compile-time choice of vertex/edge and
 * sync/async code (Sec. 2 "flexible processing": edge-based code for skewed
 * degrees, vertex-based for near-uniform ones, worklists for long
 * propagation; Sec. 4.3): a plan for this graph and algorithm -- the mode,
 * the persistent CTAs per SM and the bucket width -- from fg_autotune's
 * measurement if it ran for the algorithm, else from a selection model on
 * two features of the graph: the skew of its out-degrees (the Gini
 * coefficient of their distribution, computed at creation) and its depth (the
 * number of BFS levels from a high-degree vertex, run once and cached on
 * first use).  The model, fitted to GB300 measurements of every mode on
 * R-MAT, grid and uniform random graphs of 2^10 to 2^24 vertices (deep = more
 * than 32 levels, skewed = Gini above 0.5):
 *   SSSP  deep: FG_BUCKET from 2^21 vertices, else FG_VERTEX_SYNC;
 *         shallow: FG_EDGE_ASYNC if skewed or from 2^19 vertices, else
 *         FG_EDGE_SYNC;
 *   BFS   deep: FG_BUCKET from 2^21 vertices, else FG_VERTEX_SYNC;
 *         shallow: FG_PULL if skewed, else FG_VERTEX_SYNC;
 *   CC    deep: FG_PULL below 2^23 vertices, else FG_VERTEX_SYNC;
 *         shallow: FG_EDGE_SYNC if not skewed or below 2^14 vertices,
 *         FG_BUCKET below 2^19, else FG_VERTEX_ASYNC;
 * with 2 CTAs per SM for graphs of at most 3 million edges (BFS: 9 million),
 * whose rounds are short enough that a grid barrier over fewer CTAs pays,
 * else the occupancy limit.  FG_AUTO runs the plan (its CTAs per SM unless
 * the caller sets blocks_per_sm).  Batches (fg_run_batch, the server) take
 * the plan's mode; their team sizes come from the batch planner.
 */
typedef struct {
    int32_t mode;               /* fg_mode to run */
    int32_t blocks_per_sm;      /* persistent CTAs per SM for it (0 = the occupancy limit) */
    int32_t delta;              /* FG_BUCKET: the bucket width it uses (0 for other modes) */
    int32_t tuned;              /* 1: mode and CTAs per SM measured by fg_autotune; 0: the model */
    int32_t depth_est;          /* the model's features: BFS levels from a high-degree vertex */
    float degree_gini;          /*   and the Gini coefficient of the out-degrees (0 uniform .. 1) */
} fg_plan;
fg_status fg_select_plan(const fg_graph *g, fg_algo algo, fg_plan *out);

/* The plan's mode (fg_select_plan). */
fg_status fg_select_mode(const fg_graph *g, fg_algo algo, fg_mode *out);

/* Options and statistics of fg_run.  Zero-initialised options mean defaults. */
typedef struct {
    void *stream;               /* cudaStream_t to run on; NULL = legacy default stream */
    int32_t max_rounds;         /* round / generation cap; 0 = n + 2 */
    int32_t wait_timeout_ms;    /* bound on any single device-side wait; 0 = 1000 ms */
    int32_t blocks_per_sm;      /* persistent CTAs per SM; 0 = occupancy limit */
    int32_t inject_missing_arrival; /* testing aid for failure detection: if nonzero, CTA 0
                                   leaves the kernel without arriving at the first grid
                                   barrier, so every other CTA's bounded wait runs out and
                                   the call returns FG_ERR_TIMEOUT (the context stays
                                   usable).  0 in normal use. */
    uint64_t *round_trace;      /* optional device buffer: CTA 0 writes %globaltimer (ns) at
                                   every grid barrier of the query (init, each round, and each
                                   mid-round or pointer-jumping barrier), at most
                                   round_trace_cap entries; NULL = no tracing */
    int32_t round_trace_cap;
    int32_t delta;              /* FG_BUCKET and fg_run_multi SSSP: bucket width (0 = 5 x the mean edge weight x the
                                   mean out-degree) */
} fg_options;

typedef struct {
    int32_t mode;               /* mode that ran (FG_AUTO resolved) */
    int32_t rounds;             /* sync rounds or async worklist generations, final
                                   no-change round included (FG_BUCKET: far-list splits
                                   included; max_rounds counts the other generations) */
    int32_t jump_passes;        /* CC pointer-jumping passes */
    int32_t grid_blocks;        /* persistent CTAs launched */
    int64_t vertices_processed; /* active vertices expanded, summed over rounds
                                   (FG_EDGE_ASYNC: worklist items expanded; its dense
                                   generations stream the edge list and count none) */
    int64_t edges_relaxed;      /* edges whose source was active, summed over rounds */
    int64_t updates;            /* successful MIN updates */
    int64_t pushes;             /* worklist appends (async modes) */
    int64_t scanned;            /* activity words read by the sync modes' scans (vertex ids,
                                   or edge sources streamed by edge-sync), and the edge
                                   sources streamed by FG_EDGE_ASYNC's dense generations,
                                   summed over rounds */
    float kernel_ms;            /* device time of the fixpoint kernel (CUDA events on
                                   the query's stream) */
    int32_t barriers;           /* grid barriers the kernel passed (= trace entries written,
                                   up to the cap) */
    int32_t pull_rounds;        /* FG_PULL: rounds that pulled over the in-neighbours */
    int64_t edges_pulled;       /* FG_PULL: in-edges read by those rounds */
} fg_stats;

/*
 * General query: algo, src (ignored for CC), out, mode, options (NULL =
 * defaults) and stats (NULL = not wanted).  Blocks until out is written or an
 * error is known.  FG_ERR_TIMEOUT if max_rounds rounds were not enough or a
 * device wait exceeded wait_timeout_ms.
 */
fg_status fg_run(const fg_graph *g, fg_algo algo, int32_t src, int32_t *out, fg_mode mode,
                 const fg_options *opt, fg_stats *stats);

/*
 * Several queries of one algorithm on one graph at once: k in [1,
 * FG_MULTI_MAX] sources srcs[k] (host array; ignored for CC; repeats are
 * allowed) and k outputs outs[k] (host array of pointers, each an int32[n]
 * in host or device memory).  Output j receives exactly what fg_run(g, algo,
 * srcs[j], ...) gives in any mode.
 *
 * SSSP runs as one multi-source sweep, the k-source form of Alg. 1:
 * vertex-based over the degree buckets, every vertex's k values in one
 * 32-byte row (one L2 sector), updated in place by atomic MIN and driven by a
 * per-vertex round stamp until a round lowers nothing.  The k sources share
 * one near-far order (the one FG_BUCKET runs for one source): values at
 * or above a threshold T wait; when a round lowers nothing below T, T moves
 * to the smallest waiting value plus the width delta, and the sweep ends when
 * nothing waits.  Each source measures from itself, so the one schedule is a
 * near-far delta-stepping for every source.  Each relaxed edge
 * reads its target id and weight once for all k sources and probes the
 * target's k values with one sector access, so k queries cost far less than
 * k separate sweeps.  BFS runs as a k-source level-synchronous sweep (Alg. 3
 * for k sources at once): one byte per vertex holds which sources have
 * reached it, the frontier of each round is a byte mask per vertex, an edge
 * claims its target for the frontier's new sources with one atomic OR, and
 * each source's level is written to its output when the source first
 * reaches the vertex.  This is the on-device form of the paper's overlap of
 * independent computations (barrier-free kernels on separate streams,
 * Sec. 3.2; independent parallel sections, Sec. 3.4) for queries that share
 * a graph.  CC has no source: it runs once (in fg_select_mode's mode) and is
 * copied to every output.
 *
 * Options: stream, max_rounds (0 = n + 2 for BFS and CC, 2 k n + 2 for
 * SSSP, whose epochs add rounds), wait_timeout_ms, blocks_per_sm, delta (the
 * SSSP width; 0 = FG_BUCKET's default, 5 x mean weight x mean out-degree);
 * the other fields are ignored.  status_out[k] (may be NULL) receives each
 * query's status: they differ only when some SSSP sources overflow
 * (FG_ERR_OVERFLOW for those, FG_OK and their outputs for the others).
 * stats (may be NULL) describes the one fused sweep (mode = -1).  Returns
 * FG_OK if every query succeeded, else the first failing status; a failing
 * SSSP query's output is untouched, while BFS writes its levels as the
 * sweep runs, so after a BFS error (a timeout) the outputs are unspecified.
 * Blocks until the outputs are written.  Device state: SSSP 40 bytes per
 * vertex (rows, stamps, far marks), BFS 4 bytes per vertex (masks), plus 4 per
 * vertex for each host output.  Errors: FG_ERR_INVALID_ARG (k outside [1,
 * FG_MULTI_MAX], NULL, a source outside [0,n), wrong device),
 * FG_ERR_OVERFLOW, FG_ERR_OUT_OF_MEMORY, FG_ERR_TIMEOUT, FG_ERR_CUDA.
 */
#define FG_MULTI_MAX 8
fg_status fg_run_multi(const fg_graph *g, fg_algo algo, int32_t k, const int32_t *srcs, int32_t *const *outs,
                       const fg_options *opt, fg_status *status_out, fg_stats *stats);

/*
 * One synchronous relaxation round with every vertex active, from caller
 * state: the topology-driven body of Alg. 1 (FG_VERTEX_SYNC, over the CSR
 * buckets) or Alg. 2 (FG_EDGE_SYNC, over the edge list) applied once, for
 * SSSP.  cur and next are device int32[n] that must not overlap; for every
 * edge u->v with cur[u] < INT32_MAX, next[v] = min(next[v], cur[u] + w).  A
 * candidate that reaches INT32_MAX is not written; the call then returns
 * FG_ERR_OVERFLOW after applying every other edge.  *updates (may be NULL)
 * receives the number of successful lowering writes, which depends on the
 * schedule: at least the number of lowered vertices, at most the number of
 * edges.  *kernel_ms (may be NULL) receives the kernel's device time.  On a
 * renumbered graph (FG_GRAPH_RELABEL) cur and next stay in original order:
 * they are gathered into internal order before the kernel and next is
 * gathered back after it (2 n int32 of device scratch; kernel_ms covers the
 * round's kernel only).  Runs
 * on `stream` (NULL: legacy default stream) and blocks until done.  Used to
 * measure the sweep against the HBM roofline.  Errors: FG_ERR_INVALID_ARG
 * (NULL, host pointers, mode not FG_VERTEX_SYNC/FG_EDGE_SYNC, another
 * device's graph), FG_ERR_OVERFLOW, FG_ERR_TIMEOUT, FG_ERR_CUDA.
 */
fg_status fg_sweep(const fg_graph *g, fg_mode mode, const int32_t *cur, int32_t *next,
                   void *stream, int64_t *updates, float *kernel_ms);

/*
 * fg_sssp_csr_noalloc -- shortest paths without any device allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc, e.g. code whose device memory is all owned by another
 * allocator (a framework's caching pool that has reserved the budget), or a
 * latency-critical loop where an allocation may synchronise the device or
 * fail.  It computes what fg_sssp computes with FG_VERTEX_SYNC, directly from
 * a caller-owned CSR:
 *   n <= FG_NOALLOC_MAX_VERTICES vertices (larger n: FG_ERR_INVALID_ARG);
 *   m < 2^31 edges (larger m: FG_ERR_INVALID_ARG);
 *   row_off[n+1] int64, col[m] int32, w[m] int32 (>= 0) or NULL for unit
 *   weights, dist_out[n] int32 -- all device memory owned by the current
 *   device (host memory, or memory of another device: FG_ERR_INVALID_ARG);
 *   stream: cudaStream_t or NULL for the legacy default stream.
 * Its scratch (a second distance buffer, two activity-stamp arrays and the
 * control block) is one fixed array of about 12 MiB in the library's device
 * image; every GPU that loads the library holds it until the process exits.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current), so make the first call before any
 * stream capture.  Every call on a device shares the one array and starts by
 * clearing its control block: calls that overlap on the GPU (another stream,
 * another host thread) race and must not be issued.  dist_out doubles as the
 * first distance buffer, so on error its contents are unspecified.  The call
 * waits for `stream` to finish its work before it returns.  Unlike fg_run,
 * its limits are fixed: every device-side wait gives up after 1 s, and the
 * round cap is n + 2 (a synchronous round count never exceeds n + 1 for
 * non-negative weights, so valid input does not reach it); FG_ERR_TIMEOUT
 * comes from either.  The CSR (offsets, ids) and the weights are validated
 * on the device before any indexed access.  Errors: FG_ERR_INVALID_ARG
 * (sizes, NULL, pointers that are not this device's memory, invalid CSR or
 * negative weight), FG_ERR_OVERFLOW, FG_ERR_TIMEOUT, FG_ERR_CUDA.
 */
#define FG_NOALLOC_MAX_VERTICES 1048576
fg_status fg_sssp_csr_noalloc(int32_t n, int64_t m, const int64_t *row_off, const int32_t *col,
                              const int32_t *w, int32_t src, int32_t *dist_out, void *stream);

/* Number of kernels this library has launched in this process so far (all
   threads and devices); lets a caller count the device work of a region. */
uint64_t fg_kernel_launches(void);

/*
 * Batches: many queries over many resident graphs in one launch per
 * (algorithm, mode) kind present, the kinds running concurrently -- the
 * runtime form of the paper's barrier-free kernels on separate streams
 * (Sec. 3.2) and independent parallel sections (Sec. 3.4).  Each launch is
 * a persistent kernel split into teams of CTAs (team size from the query's
 * edge count, CTA share from its estimated work); teams pull queries from
 * size-class queues and run each fixpoint with a team-local barrier.
 * Results are identical to fg_run's.
 */
typedef struct {
    const fg_graph *g;          /* graph on the current device */
    int32_t algo;               /* fg_algo */
    int32_t src;                /* source vertex (ignored for CC) */
    int32_t *out;               /* int32[n] result, host or device memory */
    int32_t mode;               /* fg_mode; FG_AUTO = fg_select_mode's choice */
} fg_query;

typedef struct {
    void *stream;               /* cudaStream_t; NULL = legacy default stream */
    int32_t use_cuda_graph;     /* nonzero: capture the launches in a CUDA graph, launch it */
    int32_t wait_timeout_ms;    /* bound on any device-side wait; 0 = 1000 ms */
    int32_t fuse_same_graph;    /* nonzero: queries on the same graph share work -- SSSP and BFS
                                   queries run as multi-source sweeps of up to FG_MULTI_MAX
                                   sources (fg_run_multi's sweep), CC queries as one computation
                                   copied to every output (a lone query runs in its own mode);
                                   results are identical, stats_out then describe the shared
                                   sweep (mode -1 for a multi-source one) */
} fg_batch_options;

typedef struct {
    float kernel_ms;            /* device time of the batch (events around all launches) */
    int32_t launches;           /* persistent kernels launched (kinds present) */
    int32_t teams;              /* teams over all launches */
    int32_t ctas;               /* CTAs over all launches */
} fg_batch_stats;

/*
 * Runs nq queries.  status_out[nq] and stats_out[nq] (each may be NULL)
 * receive every query's outcome and counters (kernel_ms is per batch, in
 * bstats).  Returns FG_OK if every query succeeded, else the first failing
 * query's status; the outputs of successful queries are written either way.
 */
fg_status fg_run_batch(const fg_query *queries, int32_t nq, const fg_batch_options *opt,
                       fg_status *status_out, fg_stats *stats_out, fg_batch_stats *bstats);

/*
 * Query server with continuous batching (no paper counterpart beyond the
 * independent-kernel overlap of Sec. 3.2; this is the serving loop around
 * the batched path).  Requests are queued by fg_server_submit from any host
 * thread; a native worker admits them in waves -- whenever one of
 * max_inflight wave slots is free and the device memory of the in-flight
 * queries' state stays within hbm_budget_bytes, the oldest pending request
 * and later ones of the same kind (graph, algorithm, mode), up to max_wave,
 * are launched together on the slot's stream -- so waves overlap on the
 * device and new requests start as soon as a slot and memory free up.
 * Requests on large graphs (exclusive_edges) run on the whole device without
 * other graphs' requests (fused with the pending requests of their graph
 * and algorithm unless no_fusion).  one_at_a_time = 1 serves the queue
 * strictly in order, one request at a time, with the plain per-query kernel
 * (the baseline).
 * A request's work is ordered after all work enqueued on the legacy default
 * stream before it was submitted (so outputs prepared there are safe); it
 * runs on the server's own streams otherwise.  Graphs must stay alive and
 * outputs untouched until their requests complete; host outputs should be
 * pinned memory (pageable memory makes the worker wait on each copy).  A
 * failed request's output is unspecified.
 */
typedef struct fg_server fg_server;

typedef struct {
    int64_t hbm_budget_bytes;   /* in-flight query state limit; 0 = 8 GiB */
    int32_t max_inflight;       /* concurrent waves; 0 = 2 */
    int32_t max_wave;           /* requests per wave at most; 0 = 64 */
    int32_t one_at_a_time;      /* nonzero: the one-query-at-a-time baseline */
    int32_t wait_timeout_ms;    /* bound on any device-side wait; 0 = 1000 ms */
    int64_t exclusive_edges;    /* a request on a graph with at least this many edges (the
                                   symmetrised count for CC) runs alone on the whole device
                                   once the waves before it finish, with the plain per-query
                                   kernel: such a query already fills the GPU, and sharing
                                   SMs with other queries costs it L1 hits; 0 = 2^25,
                                   < 0 = never */
    int32_t no_fusion;          /* 0 (default): requests on the same graph share work -- a
                                   large-graph request runs together with the later pending
                                   requests of its graph and algorithm (up to FG_MULTI_MAX
                                   SSSP or BFS requests as one multi-source sweep, every
                                   pending CC request as one computation copied to each
                                   output), and waves on smaller graphs are fused the same way
                                   (fg_batch_options.fuse_same_graph); results are identical
                                   and fg_completion.wave_size counts the requests served
                                   together.  Nonzero: every request runs its own fixpoint in
                                   its own mode */
} fg_server_options;

typedef struct {
    uint64_t ticket;            /* as returned by fg_server_submit */
    int32_t status;             /* fg_status of the request */
    int32_t wave_size;          /* requests in the wave it ran in */
    double latency_ms;          /* submission to completion */
} fg_completion;

fg_status fg_server_create(const fg_server_options *opt, fg_server **out);
/* Queues one request (FG_AUTO is resolved here); *ticket identifies it. */
fg_status fg_server_submit(fg_server *s, const fg_query *q, uint64_t *ticket);
/* Moves up to cap completions (any order) into out; returns how many. */
int32_t fg_server_poll(fg_server *s, fg_completion *out, int32_t cap);
/* Waits until every submitted request has completed (timeout_ms 0 = no limit). */
fg_status fg_server_drain(fg_server *s, int32_t timeout_ms);
/* Serves what is queued, stops the worker and frees the server. */
fg_status fg_server_destroy(fg_server *s);

/*
 * Autotuner: times the candidate modes on this graph (queries from src,
 * ignored for CC) -- the four paper modes, FG_PULL for BFS (whose bottom-up
 * levels lower the total work) and FG_BUCKET, each at the occupancy limit and
 * at 2 CTAs per SM, the median of three runs -- writes each mode's best
 * device time in ms to times_ms[7] indexed by mode (0 for a mode not timed,
 * and for FG_AUTO; times_ms may be NULL) and the fastest mode to *best, and
 * caches it with its CTAs per SM on the handle: fg_select_plan (and
 * fg_select_mode, FG_AUTO) return the measured choice from then on.
 */
fg_status fg_autotune(const fg_graph *g, fg_algo algo, int32_t src, fg_mode *best, float *times_ms);

/* Message of the last failed call on this thread ("" if none). */
const char *fg_last_error(void);
/* Name of a status code. */
const char *fg_status_string(fg_status s);

#ifdef __cplusplus
}
#endif

#endif /* FG_H */
