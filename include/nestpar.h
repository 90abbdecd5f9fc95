/*
 * nestpar.h: C ABI of a GB300 (sm_103a) library for irregular nested-parallel
 * work, following "A Compiler Framework for Optimizing Dynamic Parallelism on
 * GPUs" (arXiv 2201.02789).
 *
 * The problem (Section II-A): each parent thread discovers a data-dependent
 * amount of nested work, N child items, and in the dynamic-parallelism form
 * launches a child grid of ceil(N / bDim) blocks with its own arguments. The
 * library runs that work in every form the paper defines:
 *
 *   no dynamic parallelism: the parent loops over its children (the "No CDP"
 *       baseline of Section VII; no launch site is compiled into that kernel);
 *   plain CDP: one device-side launch per parent (Section II-A);
 *   thresholding: launch only when N >= threshold, else run the children
 *       serially in the parent thread (Section III);
 *   coarsening: each child block runs `cfactor` consecutive original child
 *       blocks of the same parent (Section IV);
 *   aggregation: the child grids of a warp, a block, a group of blocks
 *       (multi-block granularity, Section V-A) or the whole parent grid
 *       (Section II-B) are combined into one grid; each aggregated child
 *       block finds its parent by a search over the scanned block counts
 *       (disaggregation, Section II-B); an aggregation threshold (Section
 *       V-B) lets small warp/block groups launch directly instead.
 *   The three transformations compose in the paper's order T -> C -> A
 *   (Section VI).
 *
 * Conventions (all entry points):
 *   - Every function returns an np_status. Argument errors are detected on
 *     the host and returned at once (NP_ERR_INVALID); nothing is enqueued then.
 *   - Arrays passed by pointer are caller-owned device memory unless the name
 *     ends in _host. They must stay valid until the work on `stream` is done.
 *     The context owns its workspace (frontiers, aggregation records, look-back
 *     tile states, the device error word and counters).
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream). If `stats` is non-NULL the call
 *     waits for the stream, fills *stats and returns the device-side status.
 *     Otherwise device-side errors are reported by the next np_sync().
 *   - Device-side errors: NP_ERR_LAUNCH (a device launch was refused, for
 *     example by the pending-launch limit; that parent's children then ran
 *     serially in the parent, so results stay exact), NP_ERR_TIMEOUT (a bounded
 *     wait in a look-back scan expired; results are not trustworthy),
 *     NP_ERR_CAPACITY (tessellation output too small).
 *   - One context serves one stream at a time: calls that overlap on the GPU
 *     through the same context race on its workspace.
 */
#ifndef NESTPAR_H
#define NESTPAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t np_status;
#define NP_OK 0
#define NP_ERR_INVALID 1      /* bad argument (null pointer, size, config field) */
#define NP_ERR_CUDA 2         /* a host-side CUDA call failed */
#define NP_ERR_NOMEM 3        /* device workspace allocation failed */
#define NP_ERR_CAPACITY 4     /* tessellation output buffer too small */
#define NP_ERR_LAUNCH 5       /* a device-side launch was refused (work ran serially) */
#define NP_ERR_TIMEOUT 6      /* a bounded device-side wait expired */
#define NP_ERR_UNSUPPORTED 7  /* the configuration is not available on this device */

/* ---- configuration (Sections III-V; the paper's _THRESHOLD/_CFACTOR macros
 *      and aggregation-granularity choice become runtime fields) ---- */
#define NP_VARIANT_NODP 0     /* parents loop over their children; no launch code (warp-tiled parent
                                 kernel; with NP_GRAN_NONE the CTA-tiled kernel of the device-launch
                                 forms with its launch code compiled out, Section VII-D) */
#define NP_VARIANT_CDP 1      /* dynamic parallelism with optional T, C and A */

#define NP_GRAN_NONE 0        /* one child grid per launching parent */
#define NP_GRAN_WARP 1        /* one aggregated grid per warp of parents */
#define NP_GRAN_BLOCK 2       /* one aggregated grid per parent block */
#define NP_GRAN_MULTIBLOCK 3  /* one aggregated grid per group of group_blocks parent blocks */
#define NP_GRAN_GRID_DEVICE 4 /* one aggregated grid per parent grid, launched by its last block */
#define NP_GRAN_GRID_HOST 5   /* one aggregated grid per parent grid, enqueued after it on the stream */

#define NP_SCAN_LOOKBACK 0    /* multi-block/grid scan by decoupled look-back (records in parent order) */
#define NP_SCAN_ATOMIC 1      /* the paper's packed 64-bit atomicAdd (records in arrival order) */

#define NP_DRIVER_AUTO 0      /* conditional-while CUDA graph when no device launch is needed, else host-replayed graph chunks */
#define NP_DRIVER_HOST 1      /* host loop: one level per launch, count read back after each (the paper's form) */
#define NP_DRIVER_CHUNK 2     /* `unroll` levels per host round trip, count read back after each chunk: a
                                 replayed CUDA graph for NODP / GRID_HOST, direct stream launches for
                                 the device-launch forms (a graph kernel node does not wait for the
                                 grids it launches from the device; a stream-launched kernel does) */
#define NP_DRIVER_WHILE 3     /* conditional-while CUDA graph (NODP and GRID_HOST only) */
#define NP_DRIVER_PERSISTENT 4 /* one cooperative kernel runs every level (NODP and GRID_HOST only):
                                  the parent phase, a grid barrier, the aggregated child phase and a
                                  grid barrier per level, in place of kernel boundaries; barrier waits
                                  are bounded (5 s, then NP_ERR_TIMEOUT) */

/* Where the children of the parents below the threshold run. The paper keeps
 * them in the parent thread (Section III-A); every form does so except
 * grid-host aggregation under a graph, chunk or host driver, where `serial`
 * chooses:
 *   NP_SERIAL_SPREAD  in the parent kernel (32-parent warp tiles), the items
 *                     of a warp's parents spread over the warp's lanes;
 *   NP_SERIAL_BLOCK   in the parent kernel (CTA tiles of parent_block
 *                     parents), the items of the tile's parents spread over
 *                     the CTA: the tile's records are staged in shared memory
 *                     and each thread finds its item's parent by a binary
 *                     search there;
 *   NP_SERIAL_PACKED  item by item in the aggregated child grid (threshold at
 *                     most 1024, else as BLOCK): the parent kernel records
 *                     them ({parent, start, N, first item}), and each child
 *                     CTA takes chunks of 1024 items, stages the chunk's
 *                     records in shared memory and searches there. */
#define NP_SMALL_PARENTS_MAX 2048

/* How a level loop forms the next frontier. Children append each vertex they
 * reach (the relaxation's or claim's atomic returns the old value to decide
 * it; one atomic per warp batch reserves the places), except with
 * sweep_parents > 0 (np_bfs / np_sssp, their _multi forms, the classes of a batch and the
 * pools of a server, whose sweeps skip the slots holding no query; grid-host
 * aggregation with NP_SERIAL_SPREAD, graph / chunk / host driver), a level with
 * at least that many parents instead has its children only reduce (a fire-and-forget atomic
 * min of the level, or of the packed distance and tag), and a sweep over the
 * vertex state after the level collects the vertices it reached, in vertex
 * order. Other calls and forms append. */

#define NP_SERIAL_SPREAD 0
#define NP_SERIAL_PACKED 1
#define NP_SERIAL_BLOCK 2

typedef struct np_config {
  int32_t variant;       /* NP_VARIANT_* */
  int32_t threshold;     /* launch iff N >= threshold (values <= 1: every parent with N >= 1);
                            INT32_MAX: never launch (Section III) */
  int32_t cfactor;       /* coarsening factor: 1, 2, 4, 8 or 16 (Section IV) */
  int32_t granularity;   /* NP_GRAN_* (Sections II-B, V-A) */
  int32_t group_blocks;  /* parent blocks per group at NP_GRAN_MULTIBLOCK (>= 1) */
  int32_t agg_threshold; /* warp/block granularity: groups with fewer launching parents
                            launch directly (Section V-B); 0 = off */
  int32_t child_block;   /* child block size bDim: multiple of 32 in [32, 1024] */
  int32_t parent_block;  /* parent block size: multiple of 32 in [64, 512] */
  int32_t scan;          /* NP_SCAN_* */
  int32_t driver;        /* NP_DRIVER_* (level loop of np_bfs / np_sssp) */
  int32_t unroll;        /* levels per graph chunk or per while-body, 1..16 */
  int32_t parent_grid;   /* persistent parent CTAs; 0 = resident capacity */
  int32_t serial;        /* NP_SERIAL_*: where the children of parents below the threshold run */
  int32_t small_parents; /* grid-host form, while driver: before the while loop and at the end
                            of each body one CTA runs whole levels itself while the frontier
                            has at most this many parents (<= NP_SMALL_PARENTS_MAX) and at
                            most 16384 children in all; 0 = off */
  int32_t sweep_parents; /* level loops: levels with at least this many parents form the
                            next frontier by a sweep (see below); 0 = every level appends */
  int32_t reserved[1];   /* must be zero */
} np_config;

/* Fills the library defaults: CDP, threshold 32, cfactor 4, grid-host
 * aggregation, atomic scan, child block 64, parent block 256, AUTO driver,
 * serial children spread over the parent warp, the small-level loop for levels
 * of up to 2048 parents, and a swept frontier after levels of 4096 parents or
 * more (smaller levels append)
 * (the best of a threshold x cfactor x child-block x scan sweep of BFS and SSSP
 * on an R-MAT scale-20 graph on GB300; the look-back scan, which keeps records
 * in parent order, is selectable and slower there because it publishes and
 * polls a fenced flag per 32-parent tile; the sweep threshold trades SSSP, 4%
 * faster, and the multi-query and batched forms, 15-70% faster, against a
 * single BFS, 3% slower than appending). */
np_status np_config_default(np_config *cfg);

/* ---- problem descriptions ---- */
typedef struct np_csr {       /* CSR digraph, device pointers */
  const int32_t *row_ptr;     /* [n + 1], non-decreasing, row_ptr[0] = 0, row_ptr[n] = m */
  const int32_t *col_idx;     /* [m], values in [0, n) */
  const uint32_t *weights;    /* [m] or NULL (required by SSSP) */
  int32_t n;                  /* vertices, >= 1 */
  int64_t m;                  /* edges, 0 <= m < 2^31 */
} np_csr;

typedef struct np_stats {     /* device-side counters of the last call */
  uint64_t levels;            /* non-empty levels / iterations run */
  uint64_t parents;           /* parent threads that ran (frontier pops) */
  uint64_t serial_parents;    /* parents with N > 0 that serialised their children */
  uint64_t launch_parents;    /* parents whose children ran in a child grid */
  uint64_t device_launches;   /* device-side kernel launches performed */
  uint64_t aggregated_grids;  /* of which aggregated child grids */
  uint64_t child_blocks;      /* coarsened child blocks executed */
  uint64_t items;             /* child items executed (edges visited/relaxed, points) */
  uint64_t pushes;            /* vertices appended to frontiers */
  uint64_t launch_failures;   /* refused device launches (serialised instead) */
  uint64_t timeouts;          /* expired bounded waits */
  uint64_t child_items;       /* of `items`, those run by child grids (not serialised) */
  uint64_t graph_iterations;  /* conditional-while body iterations (while driver) */
  uint32_t error;             /* device error bits: 1 launch, 2 timeout, 4 capacity */
  uint32_t reserved;
} np_stats;

typedef struct np_ctx np_ctx;

/* Creates a context on `device` (made current for the calls that use it).
 * Raises the device-runtime pending-launch limit to what plain CDP needs. */
np_status np_create(np_ctx **out, int32_t device);
np_status np_destroy(np_ctx *ctx);

/* Bytes of device workspace a call with up to `max_parents` parents per level
 * needs under `cfg` (the context allocates it on first use and keeps it). */
np_status np_workspace_size(int64_t max_parents, const np_config *cfg, size_t *bytes);

/* Waits for `stream`, returns the sticky device-side status of the context
 * (and clears it) and, if `stats` is non-NULL, the counters of the last call. */
np_status np_sync(np_ctx *ctx, void *stream, np_stats *stats);

/* Breadth-first search from `src` (Section VII, BFS benchmark): level[v] =
 * hop distance from src, -1 if unreachable; level is fully overwritten.
 * Parent = frontier vertex u, N = out-degree of u, child item = edge u->v,
 * which claims v (level -1 -> L+1) and appends it to the next frontier. */
np_status np_bfs(np_ctx *ctx, const np_csr *g, int32_t src, int32_t *level,
                 const np_config *cfg, void *stream, np_stats *stats);

/* Single-source shortest paths from `src` by frontier Bellman-Ford (Section
 * VII, SSSP benchmark): dist[v] = least uint32 weight sum, UINT32_MAX if
 * unreachable. Child item = edge relaxation by atomic minimum; an improved
 * vertex joins the next frontier once per iteration. Path sums must stay
 * below 2^32 - 1. */
np_status np_sssp(np_ctx *ctx, const np_csr *g, int32_t src, uint32_t *dist,
                  const np_config *cfg, void *stream, np_stats *stats);

/* ---- several traversals of one graph in one level loop ----
 * nsrc queries from sources[q] (host array) on the same graph. Query q's
 * vertices are ids q*ld + v, so the frontiers of all queries form one parent
 * set per level and their children aggregate into the same child grids
 * (Section V's aggregation, applied across queries). Row q of level / dist
 * (device, nsrc*ld elements, row stride ld) receives query q's result as
 * np_bfs / np_sssp define it; elements n..ld-1 of a row are left unreached
 * (a swept frontier, sweep_parents > 0, sweeps all nsrc*ld elements).
 * ld must be a power of two >= n with nsrc*ld < 2^31. The workspace scales
 * with nsrc*ld (about 36 bytes per element). */
np_status np_bfs_multi(np_ctx *ctx, const np_csr *g, int32_t nsrc, const int32_t *sources,
                       int32_t *level, int64_t ld, const np_config *cfg, void *stream,
                       np_stats *stats);
np_status np_sssp_multi(np_ctx *ctx, const np_csr *g, int32_t nsrc, const int32_t *sources,
                        uint32_t *dist, int64_t ld, const np_config *cfg, void *stream,
                        np_stats *stats);

/* ---- batched solves: many independent instances in one graph launch ----
 * (The paper runs one instance at a time; batching applies its aggregation
 * across instances.) np_batch_create copies `count` device CSR graphs
 * (graphs[i] a host array of descriptors) into per-group disjoint unions:
 * instances are grouped into size classes by floor(log2 n), `class_log2_width`
 * powers of two per class, and a class is split into groups of at most
 * `max_group_edges` edges. A group is solved as one multi-source traversal of
 * its union graph (its components are disjoint, so every instance gets
 * exactly its own result). np_batch_run launches one CUDA graph in which every
 * group is a parallel branch: unreached fill, source seeding, and a
 * conditional-while level loop. Only forms without device-side launches can
 * sit in a conditional body: NP_VARIANT_NODP, or NP_VARIANT_CDP with
 * NP_GRAN_GRID_HOST (others get NP_ERR_UNSUPPORTED). The batch owns its union
 * copies (device memory about the inputs' size) and workspaces; the inputs
 * may be freed after np_batch_create returns. np_batch_create first waits
 * for the device (the inputs may come from any stream), then checks every
 * graph on the GPU (row_ptr[0] = 0, non-decreasing, row_ptr[n] = m, column
 * indices in [0, n)) and returns NP_ERR_INVALID if one breaks that. */
#define NP_BATCH_BFS 0
#define NP_BATCH_SSSP 1
typedef struct np_batch_options {
  int32_t kind;               /* NP_BATCH_BFS or NP_BATCH_SSSP */
  int32_t class_log2_width;   /* powers of two of n per size class (0 = 2) */
  int64_t max_group_edges;    /* a group holds one instance, or several with at most
                               * this many edges in total (0 = 2^30; < 2^31) */
  np_config config;           /* initial configuration of every class */
} np_batch_options;

typedef struct np_batch_class {
  int32_t log2_lo;            /* instances with floor(log2 n) in [log2_lo, log2_lo + width) */
  int32_t instances;
  int32_t groups;
  int32_t reserved;
  int64_t vertices;
  int64_t edges;
  np_config config;           /* configuration in use */
  double tuned_ms;            /* the class's time under `config` when tuned (0 = not tuned) */
  int32_t candidates;         /* configurations the tuner timed */
  int32_t reserved2;
  /* The tuner's device-launch candidates (granularity block, multi-block of 8
   * parent blocks or grid-device, threshold 32 or 512, cfactor 4), timed on the
   * class as stream-ordered launches outside the batch graph: a graph kernel
   * node does not wait for the grids it launches from the device, so these
   * forms cannot run inside the one-launch batch. The fastest of them: */
  double device_launch_ms;    /* its time (0 = not measured) */
  int32_t device_launch_granularity;   /* its NP_GRAN_* */
  int32_t device_launch_threshold;     /* its threshold */
} np_batch_class;

typedef struct np_batch np_batch;

/* sources: host [count], 0 <= sources[i] < graphs[i].n. SSSP needs weights. */
np_status np_batch_create(np_ctx *ctx, int32_t count, const np_csr *graphs, const int32_t *sources,
                          const np_batch_options *opt, np_batch **out);
np_status np_batch_destroy(np_batch *b);
/* Result layout: vertex v of instance i is out[offsets[i] + v]; total elements. */
np_status np_batch_layout(const np_batch *b, int64_t *offsets, int64_t *total);
np_status np_batch_classes(const np_batch *b, np_batch_class *out, int32_t max, int32_t *nclasses);
np_status np_batch_set_config(np_batch *b, int32_t cls, const np_config *cfg);
/* Autotuner (Section VII-C tunes threshold, coarsening and granularity). For
 * each class, runs the class's groups alone under each candidate configuration
 * (no dynamic parallelism; grid-host aggregation with threshold T in {8, 32,
 * 128, 512}, coarsening factor in {2, 8} and child block in {32, 128}), `reps`
 * times each (0 = 3), and keeps the configuration with the least minimum time;
 * then the kept one with a swept frontier (sweep_parents 1), kept if faster.
 * It also times the device-launch granularities (see np_batch_class), which
 * it reports but cannot pick. `out` (device, total elements) is overwritten. */
np_status np_batch_tune(np_batch *b, void *out, int32_t reps, void *stream);
/* Solves every instance into `out` (device int32 levels or uint32 distances,
 * total elements). stats (nullable, waits) are summed over groups. */
np_status np_batch_run(np_batch *b, void *out, void *stream, np_stats *stats);

/* ---- serving: continuous batching of traversal queries ----
 * (The paper has no serving layer.) A server keeps `ngraphs` device graphs
 * resident (the caller keeps them alive) and one pool per (graph, kind).
 * A pool holds S query slots: per-slot level or distance arrays of
 * npad = next power of two >= n elements, and one level loop whose frontier
 * holds the vertices (slot*npad + v) of every query in the pool, so the
 * queries' children aggregate into the same grids. Memory-based admission:
 * the budget is divided evenly over the pools and each pool gets
 * S = min(max_slots, share / bytes_per_slot) slots (NP_ERR_NOMEM if a pool
 * gets none). np_server_submit only queues a query. np_server_step, for
 * every pool with work: admits queued queries into free slots (between
 * levels: the slot is reset and its source joins the current frontier),
 * runs `levels_per_step` levels, counts each slot's frontier entries and
 * copies finished queries (no entries left) to their `out` arrays, all as
 * one CUDA graph per pool on the pool's own stream, so pools overlap on the
 * device; then it waits and marks finished queries done. Results equal
 * np_bfs / np_sssp from the same source. np_server_create waits for the
 * device and checks every graph as np_batch_create does. An `out` array must
 * not be touched by other work until its query is done. */
typedef struct np_server_options {
  uint64_t memory_budget;     /* bytes for slot state (0 = a quarter of free device memory) */
  int32_t max_slots;          /* per pool (0 = 64) */
  int32_t levels_per_step;    /* 0 = 2 */
  np_config bfs_config;       /* forms without device-side launches only */
  np_config sssp_config;
} np_server_options;

typedef struct np_query_info {
  int32_t done;               /* 1 once `out` holds the result */
  int32_t graph;
  int32_t kind;               /* NP_BATCH_BFS or NP_BATCH_SSSP */
  int32_t slot;               /* -1 while queued */
  int64_t submit_step;        /* server step counter at submission, admission, completion */
  int64_t admit_step;
  int64_t finish_step;
} np_query_info;

typedef struct np_server np_server;

np_status np_server_create(np_ctx *ctx, const np_csr *graphs, int32_t ngraphs,
                           const np_server_options *opt, np_server **out);
np_status np_server_destroy(np_server *s);
/* Slots and bytes per slot of pool (graph, kind). */
np_status np_server_pool_info(const np_server *s, int32_t graph, int32_t kind, int32_t *slots,
                              uint64_t *bytes_per_slot);
/* Queues a query; out is a device array of graphs[graph].n int32 levels (BFS)
 * or uint32 distances (SSSP), written when the query finishes. */
np_status np_server_submit(np_server *s, int32_t graph, int32_t kind, int32_t src, void *out,
                           int64_t *ticket);
/* One serving round (see above). *in_flight = queries queued or resident after it. */
np_status np_server_step(np_server *s, int32_t *in_flight);
np_status np_server_poll(const np_server *s, int64_t ticket, np_query_info *info);
/* Moves up to `max` tickets of queries finished since the last call (oldest
 * first) into tickets[]; *count = how many. */
np_status np_server_finished(np_server *s, int64_t *tickets, int32_t max, int32_t *count);

/* Quadratic Bezier tessellation (Section VII, BT benchmark). ctrl is
 * float[ncurves][3][2]. Parent = curve c with curvature
 * kappa = |P0 - 2P1 + P2| / |P2 - P0| and N = clamp(ceil(sqrt(kappa)*64), 4, 4096)
 * (computed in FP64 with correctly rounded operations; zero chord: 4096 if the
 * second difference is non-zero, else 4). offsets[0..ncurves] receives the
 * curve-order exclusive scan of N (offsets[ncurves] = total). Child item j
 * writes points[offsets[c] + j] = B(j / (N - 1)) in FP32. If the total
 * exceeds `cap`, curves that do not fit are skipped and NP_ERR_CAPACITY is
 * reported; offsets are always complete. */
np_status np_bezier(np_ctx *ctx, const float *ctrl, int32_t ncurves, int32_t *offsets,
                    float *points, int64_t cap, const np_config *cfg, void *stream,
                    np_stats *stats);

/* Triangle counting, the second CSR workload on the same engine (Section VII's
 * nested-parallel pattern with an adjacency-intersection child). `dag` is an
 * acyclic orientation of a simple undirected graph: every undirected edge
 * appears once, from one endpoint to the other, with sorted out-lists N+ and
 * no self-loops or duplicates. Parent = vertex u, N = |N+(u)|, child item =
 * out-edge u -> v, which counts the w in both N+(u) and N+(v) (the shorter
 * list is walked, the longer binary-searched). *count (device uint64)
 * receives the number of triangles. Every form (NODP, plain CDP, T, C, A at
 * every granularity) runs one pass over the n parents. */
np_status np_triangles(np_ctx *ctx, const np_csr *dag, uint64_t *count, const np_config *cfg,
                       void *stream, np_stats *stats);

/* ---- allocation-free tessellation (the paper has no counterpart) ----
 * Some callers cannot allocate device memory at the time they call this
 * library: programs whose device memory all belongs to their own pool
 * allocator or to a budget fixed at start-up, and latency-critical loops where
 * an allocation may wait for the device. np_bezier_noalloc serves them: the
 * same tessellation as np_bezier (the kernels np_bezier runs for `cfg`, the
 * same results), with no context and no allocation of any kind. Its scratch
 * (level state, aggregation records, look-back tile states) is one static
 * device array of about 1.5 MB inside the library, sized for
 * NP_NOALLOC_MAX_CURVES curves; every GPU that loads the library holds it
 * until the process exits.
 *   - ncurves > NP_NOALLOC_MAX_CURVES is rejected with NP_ERR_INVALID before
 *     anything is enqueued; so are the argument errors of np_bezier
 *     (np_config checks included).
 *   - Only forms without device-side launches run here: NP_VARIANT_NODP, or
 *     NP_VARIANT_CDP with NP_GRAN_GRID_HOST and serial children in the parent
 *     kernel (NP_SERIAL_SPREAD or NP_SERIAL_BLOCK); other forms get
 *     NP_ERR_UNSUPPORTED.
 *   - The first call on a device looks up the array's device address and
 *     clears the array with an asynchronous memset on `stream`; make that
 *     first call before any stream capture. The address is kept for the life
 *     of the process: after cudaDeviceReset the entry point must not be used.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call resets what must start at zero. Calls that overlap on the GPU (on
 *     different streams, or from several host threads) race on the array and
 *     must be serialised by the caller.
 *   - The call only enqueues work on `stream`; it returns no stats. Its
 *     outcome is in offsets[ncurves] once the stream reaches it: the total
 *     point count; > cap when the capacity falls short (curves that do not fit
 *     are skipped); -1 when a bounded device-side wait gave up (the offsets
 *     are then not to be used). */
#define NP_NOALLOC_MAX_CURVES 65536
np_status np_bezier_noalloc(const float *ctrl, int32_t ncurves, int32_t *offsets, float *points,
                            int64_t cap, const np_config *cfg, void *stream);

/* ---- one nesting pass over an explicit parent set (Section II-A) ---- */
#define NP_COUNT_CSR_DEGREE 0   /* N = row_ptr[p+1] - row_ptr[p], child i -> edge row_ptr[p] + i */
#define NP_COUNT_BEZIER 1       /* N = the tessellation point count of curve p */
#define NP_BODY_BFS_VISIT 0     /* claim col[e] with level next_level, append it to `next` */
#define NP_BODY_SSSP_RELAX 1    /* atomic-min relax col[e]; append improved targets once per `iteration` */
#define NP_BODY_BEZIER_EVAL 2   /* write point i of curve p at points[offsets-scan + i] */
#define NP_BODY_TRIANGLES 3     /* count |N+(p) cap N+(col[e])| into tri_counts (CSR count) */

typedef struct np_parents {
  const int32_t *ids;     /* device [count] parent ids, or NULL for ids 0..count-1 */
  int32_t count;          /* >= 0 */
} np_parents;

typedef struct np_body {
  int32_t kind;           /* NP_BODY_* (must match the count kind: CSR for BFS/SSSP) */
  int32_t next_level;     /* BFS: level written to newly claimed vertices */
  int32_t iteration;      /* SSSP: stamp value of this pass (>= 1, distinct per pass) */
  int32_t reserved;
  int32_t *level;         /* BFS: [n] device */
  uint32_t *dist;         /* SSSP: [n] device */
  int32_t *stamp;         /* SSSP: [n] device, last pass that appended each vertex */
  int32_t *next;          /* BFS/SSSP: [n] device, appended vertices */
  int32_t *next_count;    /* BFS/SSSP: device int, incremented by the appends */
  const float *ctrl;      /* Bezier: [count][3][2] device (indexed by parent id) */
  int32_t *offsets;       /* Bezier: [count + 1] device, written (exclusive scan in parent order) */
  float *points;          /* Bezier: [cap][2] device */
  int64_t cap;            /* Bezier: capacity of points in points */
  uint64_t *tri_counts;   /* triangles: [NP_TRI_SLOTS] device partial counts, added to */
} np_body;
#define NP_TRI_SLOTS 256

/* Runs the children of every parent once, in the form `cfg` selects. For CSR
 * counts `g` describes the graph; for Bezier counts `g` may be NULL. */
np_status np_run_nested(np_ctx *ctx, const np_parents *parents, int32_t count_kind,
                        const np_csr *g, const np_body *body, const np_config *cfg,
                        void *stream, np_stats *stats);

/* ---- end to end from host memory: copies inputs in and results out on
 *      `stream` (pageable or pinned host buffers), waits, returns the status ---- */
np_status np_bfs_host(np_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr_host,
                      const int32_t *col_idx_host, int32_t src, int32_t *level_host,
                      const np_config *cfg, void *stream, np_stats *stats);
np_status np_sssp_host(np_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr_host,
                       const int32_t *col_idx_host, const uint32_t *weights_host, int32_t src,
                       uint32_t *dist_host, const np_config *cfg, void *stream, np_stats *stats);

/* Stream-ordered forms of np_bfs_host / np_sssp_host: they enqueue the copies in,
 * the solve and the copy out on `stream` and return without waiting. The host
 * buffers must stay valid, and the inputs unchanged, until the stream has passed
 * the call; the result is in `level_host` / `dist_host` from then on. Only
 * page-locked host buffers (cudaHostAlloc, cudaHostRegister) let the copies run
 * asynchronously; with pageable memory the runtime copies synchronously. The
 * staging buffers belong to the context, so calls on one context must be
 * ordered on one stream; two contexts on two streams let one call's copies
 * overlap the other's solve. Argument errors return synchronously, as for the
 * waiting forms; device errors are reported by the next np_sync on the context. */
np_status np_bfs_host_async(np_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr_host,
                            const int32_t *col_idx_host, int32_t src, int32_t *level_host,
                            const np_config *cfg, void *stream);
np_status np_sssp_host_async(np_ctx *ctx, int32_t n, int64_t m, const int32_t *row_ptr_host,
                             const int32_t *col_idx_host, const uint32_t *weights_host, int32_t src,
                             uint32_t *dist_host, const np_config *cfg, void *stream);

/* ---- execution-time breakdown (the paper's Section VII-B, measured instead of
 *      obtained by deactivating code) ---- */
#define NP_PROFILE_LEVELS 64
typedef struct np_profile {
  double parent_ms;           /* summed CUDA-event time of parent-grid launches */
  double child_ms;            /* summed time of stream-ordered child grids (grid-host form) */
  double other_ms;            /* init and level-advance kernels */
  int64_t parent_launches;
  int64_t child_launches;
  int64_t other_launches;
  /* per level of the last profiled np_bfs / np_sssp call (first NP_PROFILE_LEVELS
   * levels); the longest level is the paper's "longest iteration" figure */
  double longest_level_ms;
  int32_t levels;
  int32_t reserved;
  int32_t level_parents[NP_PROFILE_LEVELS];   /* frontier size of each level */
  double level_parent_ms[NP_PROFILE_LEVELS];
  double level_child_ms[NP_PROFILE_LEVELS];
} np_profile;

/* While enabled (on != 0), np_bfs / np_sssp / np_bezier / np_run_nested launch
 * every kernel of the path separately on the caller's stream (no graphs),
 * bracket each with CUDA events and wait after each level; the grids and
 * kernels are the ones the graph drivers run. Device-side (child) launches are
 * included in their parent grid's time. */
np_status np_profile_enable(np_ctx *ctx, int32_t on);
/* Accumulated times since the last reset; reset != 0 clears them. */
np_status np_profile_read(np_ctx *ctx, np_profile *out, int32_t reset);

/* Tessellation end to end: ctrl_host in, offsets_host[ncurves + 1] and
 * points_host[cap][2] out. */
np_status np_bezier_host(np_ctx *ctx, const float *ctrl_host, int32_t ncurves, int32_t *offsets_host,
                         float *points_host, int64_t cap, const np_config *cfg, void *stream,
                         np_stats *stats);

/* Checks the bounded device-side waits: runs one wait on a flag that nothing
 * sets and returns the status it ends with, which must be NP_ERR_TIMEOUT (the
 * error word is cleared afterwards and the context stays usable).
 *   which = 0: a decoupled look-back (Section V-A's multi-block scan) whose
 *              predecessor tile never publishes; gives up after its poll limit
 *              (about a second); limit_ns is ignored.
 *   which = 1: the persistent level loop's grid barrier, launched
 *              cooperatively with two CTAs of which one never arrives; gives up
 *              after limit_ns (1 ms .. 10 s).
 * Nothing faults, traps or hangs. */
np_status np_selftest_wait(np_ctx *ctx, int32_t which, int64_t limit_ns, void *stream);

const char *np_status_string(np_status s);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t np_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NESTPAR_H */
