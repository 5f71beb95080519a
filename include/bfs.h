/*
 * bfs.h -- C ABI of the GB300 breadth-first search library (libbfs_gb300.so).
 *
 * The library computes level-synchronous BFS on an undirected, unweighted graph
 * G = (V, E) (Sec. 2.1 of Buluc & Madduri, "Parallel Breadth-First Search on
 * Distributed Memory Systems").  Each level is one sparse matrix-sparse vector
 * product over the (select2nd, max) semiring, masked by the vertices already
 * reached (Sec. 3.2, Algorithm 3): with frontier values equal to the vertices'
 * own ids, a newly reached vertex takes as parent its LARGEST-id neighbour in
 * the previous frontier, which makes the BFS tree unique.
 *
 * Outputs of every traversal, for a source s:
 *   level[v]  = d(s, v), the hop distance (Algorithm 1's d), or -1 if v is not
 *               reachable from s;
 *   parent[v] = s for v = s; the largest-id neighbour u of v with
 *               level[u] = level[v] - 1 otherwise; -1 if v is not reachable
 *               (Algorithm 3's output pi).
 *
 * Conventions for every entry point:
 *   - Vertex ids are int32 in [0, n); CSR row offsets are int64 (the directed
 *     entry count of a large graph exceeds 2^31).
 *   - Pointers are DEVICE pointers (cudaMalloc or torch CUDA memory on the
 *     current device) unless a BFS_HOST_PTRS flag says otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously on it; results are valid once the stream
 *     has reached the work (synchronise it, or call bfs_sync).
 *   - Every call returns a bfs_status; on failure bfs_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *   - A graph is immutable after creation.  Runs on one graph from different
 *     host threads must use different streams; each stream gets its own
 *     workspace, created on first use and kept until bfs_graph_destroy.
 */
#ifndef BFS_GB300_H
#define BFS_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define BFS_API __attribute__((visibility("default")))
#else
#define BFS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bfs_status {
  BFS_OK = 0,
  BFS_ERR_INVALID_ARG = 1,   /* bad source, NULL pointer, size out of range */
  BFS_ERR_INVALID_GRAPH = 2, /* BFS_VALIDATE found a malformed CSR */
  BFS_ERR_OOM = 3,           /* a device allocation failed */
  BFS_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the CUDA error) */
  BFS_ERR_TIMEOUT = 5,       /* a device-side wait hit its iteration limit; the run was abandoned */
  BFS_ERR_UNSUPPORTED = 6,   /* no CUDA device, or a device older than sm_103 */
  BFS_ERR_BOUNDS = 7         /* bounds-checking build only: an index outside its array (see below) */
} bfs_status;

/*
 * The bounds-checking build (the same sources compiled with -DBFS_BOUNDS_CHECK,
 * shipped beside the normal library as libbfs_gb300_checked.so) checks every
 * index the traversal kernels take from the graph or from a counter before
 * using it: each adjacency id against [0, n), each frontier-queue slot against
 * n, each chunk-list slot against the list's capacity.  An index outside its
 * range is not used; the first one is recorded with its site, and the call
 * that reports the device status (bfs_sync, a synchronising run, the ragged
 * or static entry points) returns BFS_ERR_BOUNDS with the site and the index
 * in bfs_last_error().  Row offsets are checked where a graph is created, and
 * by each bfs_run_static call (non-decreasing from 0 to nnz; BFS_ERR_BOUNDS
 * otherwise), even without BFS_VALIDATE.  The normal build has none of these
 * checks.  Results of a well-formed graph are identical in both builds.
 */
BFS_API int bfs_bounds_checked(void); /* 1 in the bounds-checking build, 0 otherwise */

/* Flags of bfs_graph_create / bfs_graph_create_from_edges / bfs_opts.flags. */
#define BFS_HOST_PTRS 0x1u /* the input (graph create) or output (run) pointers are host memory */
#define BFS_VALIDATE 0x2u  /* graph create: check the CSR on the device before accepting it */
#define BFS_DIRECTED 0x4u  /* graph create: the arcs are directed (see below) */
#define BFS_HOST_ASYNC 0x8u /* bfs_run with BFS_HOST_PTRS: return once the copies are enqueued (see bfs_run) */

/* Per-level expansion variants (each gives identical levels and parents). */
typedef enum bfs_variant {
  BFS_VARIANT_TD_THREAD = 0, /* top-down SpMSV, one thread per frontier vertex */
  BFS_VARIANT_TD_WARP = 1,   /* top-down SpMSV, one warp per frontier vertex */
  BFS_VARIANT_TD_BINNED = 2, /* top-down SpMSV, thread / warp / CTA per vertex by degree bin */
  BFS_VARIANT_PULL = 3,      /* dense-frontier SpMV: unvisited rows scan their adjacency, largest id first */
  BFS_VARIANT_TILED = 4,     /* dense-frontier SpMV over the 2D tiles of Sec. 3.2 stored as DCSC (Sec. 4.1),
                                with tile-local frontier and row slices in shared memory (bfs_graph_tiles) */
  BFS_NUM_VARIANTS = 5
} bfs_variant;

/* How bfs_run picks the variant of each level. */
typedef enum bfs_selector {
  BFS_SELECT_HEURISTIC = 0, /* fixed thresholds on frontier / unvisited edge counts */
  BFS_SELECT_LEARNED = 1,   /* the selector network set by bfs_selector_set_params (heuristic if none) */
  BFS_SELECT_FORCED = 2,    /* opts.forced_variant at every level */
  BFS_SELECT_SCHEDULE = 3   /* opts.schedule[k] at level k (the heuristic beyond schedule_len) */
} bfs_selector;

/* Statistics of one level k of a traversal (filled when bfs_opts.stats != NULL). */
typedef struct bfs_level_stat {
  int64_t frontier_count;   /* |f_k| */
  int64_t frontier_edges;   /* sum of the degrees of f_k */
  int64_t bin_count[3];     /* vertices of f_k with degree <= 32, <= 1024, larger */
  int64_t unvisited_count;  /* vertices not reached before level k+1 starts: n - sum_{i<=k} |f_i| */
  int64_t unvisited_edges;  /* nnz - sum_{i<=k} sum deg f_i */
  int64_t time_ns;          /* device time of level k (global timer, between grid barriers) */
  int32_t variant;          /* bfs_variant used to expand level k */
  int32_t reserved;
} bfs_level_stat;

/* Tuning knobs (bfs_autotune fills them; zero fields mean "library default"). */
typedef struct bfs_tuning {
  int32_t warp_degree;   /* TD_BINNED: degree from which a vertex gets a warp (default 32) */
  int32_t cta_degree;    /* TD_BINNED: degree from which a vertex gets a CTA (default 256) */
  int32_t pull_thread_degree; /* PULL: top entries of a row each lane tests alone before the warp-wide scan
                                 (1..4, larger values act as 4; default 4) */
  int32_t chunk_degree;  /* top-down: vertices above this degree are split into grid-wide chunks of 1024
                            edges (>= 1024, default 1024) */
  float alpha;           /* heuristic: go PULL when frontier edges * alpha' > unvisited edges and the
                            frontier grows, alpha' = alpha * (1 + 4 n / L2 bytes) (default 20) */
  float beta;            /* heuristic: leave PULL when frontier count < n / beta (default 24) */
  int32_t batch_topdown_limit; /* batched: levels with at most this many active vertices expand top-down (default n/64) */
  int32_t small_frontier; /* heuristic: a top-down level whose frontier has at most this many vertices, none of
                             degree above 32, runs TD_WARP instead of TD_BINNED (0 = default: the warps resident
                             in the traversal's grid; negative = never) */
  int32_t batch_width;   /* batched: roots per traversal, the bits of a frontier word: 8, 16, 32 or 64
                            (default 64) */
  int32_t narrow_edges;  /* a level whose frontier has at most this many edges runs on half the CTAs of the
                            traversal's grid, which also halves its barrier's arrivals (0 = default 16384;
                            negative = never) */
  int32_t ctas_per_sm;   /* single-root traversals: CTAs per SM in the persistent grid (0 = default: as many as
                            fit, two; 1 = one; larger values act as the default).  One CTA per SM halves
                            every barrier's arrivals and suits graphs of many small levels (3D grid 128^3:
                            14 % faster) but leaves half the warps of a large level's latency hiding unused
                            (R-MAT scale 26: 40 % slower) */
} bfs_tuning;

/* Options of one run (NULL = heuristic selector, no statistics). */
typedef struct bfs_opts {
  int32_t selector;          /* bfs_selector */
  int32_t forced_variant;    /* BFS_SELECT_FORCED */
  const int32_t* schedule;   /* BFS_SELECT_SCHEDULE: host array of schedule_len variants */
  int32_t schedule_len;
  int32_t max_stat_levels;   /* capacity of `stats` (levels beyond it are not recorded) */
  bfs_level_stat* stats;     /* host array; when set, the call synchronises the stream */
  int32_t* nlevels_out;      /* host int; when set, the call synchronises and writes the level count */
  int64_t* edges_out;        /* host int64; when set, the call synchronises and writes the TEPS edge
                                count of the traversal (undirected edges inside the reached set) */
  uint32_t spin_limit;       /* device wait limit in polls (0 = default, about one second) */
  uint32_t flags;            /* BFS_HOST_PTRS: parent_out/level_out are host memory;
                                BFS_HOST_ASYNC with it: bfs_run does not wait for the copies */
} bfs_opts;

typedef struct bfs_graph bfs_graph;

/*
 * Graph from a CSR of an undirected graph (Sec. 4.1: rows sorted, each edge
 * stored in both rows).  offsets: int64[n+1], adj: int32[nnz], nnz = offsets[n].
 * The library copies both arrays into memory it owns; the caller keeps its
 * inputs.  With BFS_VALIDATE the copy is checked on the device (offsets
 * monotone from 0 to nnz, ids in range, rows strictly ascending, no
 * self-loops, symmetric) and BFS_ERR_INVALID_GRAPH is returned if it fails.
 * Without it, a CSR whose offsets are non-decreasing from 0 to nnz and whose
 * ids lie in [0, n) but that breaks the other rules (order, repeats, loops,
 * symmetry) gives unspecified but memory-safe results; offsets or ids outside
 * those ranges may read out of bounds (the bounds-checking build turns them
 * into BFS_ERR_BOUNDS instead).  Requires 1 <= n < 2^31 - 1 and
 * 0 <= nnz < 2^40.
 *
 * With BFS_DIRECTED the CSR holds the arcs of a directed graph: row u lists the
 * heads v of the arcs u -> v (sorted, no repeats, no self-loops; symmetry is
 * not required).  Every traversal then follows the arcs: level[v] is the
 * length of the shortest directed path s -> v and parent[v] the largest id u
 * with an arc u -> v and level[u] = level[v] - 1 (the product with A^T of
 * Sec. 3.2 when A is not symmetric).  The library also builds the transpose
 * on the device (about 8 bytes per arc more), which the pull variant scans;
 * the TEPS count (bfs_opts.edges_out) is the number of arcs leaving reached
 * vertices.  Directed graphs cannot be parts of bfs_graph_union
 * (BFS_ERR_UNSUPPORTED); bfs_graph_csr and bfs_graph_copy_csr give the
 * out-rows.
 */
BFS_API int bfs_graph_create(const int64_t* offsets, const int32_t* adj, int32_t n, int64_t nnz,
                     uint32_t flags, bfs_graph** out);

/*
 * Graph from an undirected edge list src/dst: int32[m] (device memory, or host
 * with BFS_HOST_PTRS).  Built on the device: self-loops dropped, both
 * directions emitted, 64-bit keys (u, v) radix-sorted, repeats removed, int64
 * row offsets from the sorted keys (the symmetrised, deduplicated input of the
 * paper's benchmark, Sec. 6).  Endpoints outside [0, n) give
 * BFS_ERR_INVALID_ARG.  Temporary device memory of about 40 bytes per edge is
 * allocated and released inside the call, which synchronises `stream`.  With
 * BFS_DIRECTED the pairs are arcs src -> dst: nothing is symmetrised, and the
 * graph is the directed graph of bfs_graph_create with BFS_DIRECTED.
 */
BFS_API int bfs_graph_create_from_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n,
                                uint32_t flags, void* stream, bfs_graph** out);

/*
 * Block-diagonal union of `count` graphs (vertex ids of part i shifted by the
 * sum of the sizes of parts 0..i-1).  The union owns a copy; the parts may be
 * destroyed afterwards.  Used by bfs_run_ragged.  Synchronises `stream`.
 */
BFS_API int bfs_graph_union(bfs_graph* const* graphs, int32_t count, void* stream, bfs_graph** out);

/* n, nnz (directed CSR entries) and, for a union, the number of parts (1 otherwise). */
BFS_API int bfs_graph_info(const bfs_graph* g, int32_t* n, int64_t* nnz, int32_t* parts);

/* Device pointers of the graph's own CSR (read-only for the caller). */
BFS_API int bfs_graph_csr(const bfs_graph* g, const int64_t** offsets, const int32_t** adj);

/* Copies the graph's CSR into caller buffers offsets_out int64[n+1] and
 * adj_out int32[nnz] (device memory, or host with BFS_HOST_PTRS).  Synchronous. */
BFS_API int bfs_graph_copy_csr(const bfs_graph* g, int64_t* offsets_out, int32_t* adj_out, uint32_t flags);

/* Frees the graph and every workspace created for it.  Synchronises the device. */
BFS_API void bfs_graph_destroy(bfs_graph* g);

/*
 * One BFS from `source` (Algorithm 3 on one GPU): writes level_out and
 * parent_out, int32[n] each, caller-allocated.  Runs as ONE persistent
 * cooperative kernel launch per traversal: every level is an expansion phase
 * followed by a grid-wide barrier, with the level count held on the device.
 * Asynchronous unless opts asks for statistics or host outputs.  Device-side
 * failures (BFS_ERR_TIMEOUT; BFS_ERR_BOUNDS in the bounds-checking build) are
 * returned by bfs_sync or by a synchronising call; until then further runs on the same stream do no work.
 * Host outputs (opts->flags BFS_HOST_PTRS): the traversal writes a device
 * staging buffer of the (graph, stream) workspace, then the library copies it
 * to the host arrays and waits.  With BFS_HOST_ASYNC as well, the call returns
 * once the copies are enqueued on a copy stream of the workspace, and the host
 * arrays are complete after bfs_sync(g, stream) (the host arrays must stay
 * valid until then; pinned memory gives the full copy bandwidth).  The
 * workspace then alternates between two staging buffers, so that the copies
 * of one traversal overlap the next traversal on the same stream.
 */
BFS_API int bfs_run(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out,
            const bfs_opts* opts, void* stream);

/*
 * BFS from k sources at once: outputs are root-major int32[k][n] (row i belongs
 * to sources[i], a host array).  Up to W roots share one traversal in which
 * every vertex carries W-bit frontier and visited bitsets (a boolean sparse
 * matrix-dense matrix product per level); parents follow the same max-id rule,
 * recovered by scanning each newly reached vertex's row from the largest id
 * down.  W = bfs_tuning.batch_width (8, 16, 32 or 64, default 64); k > W
 * runs in chunks of W.  Results equal k calls of bfs_run.
 * Each level expands top-down when its frontier has at most
 * bfs_tuning.batch_topdown_limit vertices, by pull otherwise.  With
 * opts->stats, the levels of the last chunk are reported (frontier_count,
 * time_ns, variant BFS_VARIANT_TD_WARP or BFS_VARIANT_PULL).
 */
BFS_API int bfs_run_batch(bfs_graph* g, const int32_t* sources, int32_t k, int32_t* parent_out,
                  int32_t* level_out, const bfs_opts* opts, void* stream);

/*
 * One traversal per part of a union graph (bfs_graph_union), all in one
 * launch: sources[i] (host array, a LOCAL id of part i) seeds part i.  Because
 * the parts are disjoint and the id shift keeps the order of ids inside a part,
 * a single multi-source BFS of the union gives every part exactly its own
 * levels and max-id parents.  parent_out[i] / level_out[i] are device arrays of
 * part i's size and receive LOCAL ids.  parent_out and level_out are host
 * arrays of `parts` device pointers.
 */
BFS_API int bfs_run_ragged(bfs_graph* u, const int32_t* sources, int32_t* const* parent_out,
                   int32_t* const* level_out, const bfs_opts* opts, void* stream);

/*
 * Single-source BFS that allocates nothing (the paper has no counterpart: this
 * entry point exists for callers of this library that cannot call cudaMalloc,
 * for example a plug-in or a real-time loop that must not trigger the device
 * synchronisation and the possible failure of an allocation, or a process
 * whose device memory was reserved up front by another allocator).
 * The caller passes the CSR (offsets int64[n+1], adj int32[nnz], device
 * memory, rows sorted, each undirected edge in both rows, not validated) and
 * the outputs parent_out / level_out (device int32[n]); results are those of
 * bfs_run with the heuristic selector.  All scratch memory of the traversal
 * (about 15.3 MB) is one static array inside the library, which every GPU that
 * loads the library holds until the process exits; hence the limits
 * n <= 1,048,576 and nnz <= 67,108,864, beyond which the call returns
 * BFS_ERR_INVALID_ARG.  The first call on a device sets up that device (looks
 * up the array's device address and clears its barrier and status words), so
 * it should come before any stream capture.  Every call zeroes the array's
 * barrier word on `stream` (a memset, no allocation) before its launch.
 * Every call shares the array and finds the previous call's contents there
 * (the traversal re-initialises what it needs), so calls that overlap on the
 * GPU race: issue one at a time per device.  Undirected graphs only (a
 * directed graph needs bfs_graph_create with BFS_DIRECTED).  The call waits for `stream` to finish the traversal and returns its
 * device status (BFS_ERR_TIMEOUT if a device-side wait reached its limit,
 * BFS_ERR_BOUNDS from the bounds-checking build).
 */
BFS_API int bfs_run_static(const int64_t* offsets, const int32_t* adj, int32_t n, int64_t nnz, int32_t source,
                           int32_t* parent_out, int32_t* level_out, void* stream);

/*
 * The 2D tiles of g that BFS_VARIANT_TILED walks: Sec. 3.2's 2D blocks of the
 * adjacency matrix, each stored in the doubly compressed sparse column form of
 * Sec. 4.1 (IR row ids indexed by the parallel arrays JC of non-empty column
 * ids and CP of column pointers).  Row blocks hold 2^rb_bits vertices v (the
 * vertices a pull level may reach), column blocks 2^cb_bits vertices u (their
 * candidate parents); tile t = rb * ncb + cb holds the entries (v, u) of v's
 * in-row (its row, for an undirected graph) with v >> rb_bits == rb and
 * u >> cb_bits == cb.  The tiles are built on the device when g has none, or
 * when rb_bits / cb_bits (each in [5, 16], or 0 for the default: cb_bits 16,
 * rb_bits so that there are about 4 row blocks per SM, within [8, 16]) differ
 * from those of g's current tiles; other values give BFS_ERR_INVALID_ARG.  A
 * traversal that uses BFS_VARIANT_TILED builds the default tiles if g has none.
 * Rebuilding must not overlap a traversal of g on another stream.  On return
 * *info holds the layout and DEVICE pointers owned by g, valid until the tiles
 * are rebuilt or g is destroyed:
 *   tdir_jc, tdir_ir (int64[ntiles + 1]): first column / first entry of tile t;
 *   jc (uint16[nzc]): tile-local ids of each tile's non-empty columns, ascending;
 *   cp (uint32[nzc]): first entry of each column relative to its tile's first
 *     entry (a column ends where the next column of its tile starts, or where
 *     its tile ends);
 *   ir (uint16[nnz]): tile-local row ids, ascending within each column.
 * Synchronises the stream.  The tiles take about 8 bytes per CSR entry.
 */
typedef struct bfs_tile_info {
  int32_t rb_bits, cb_bits; /* log2 of the rows / columns per tile */
  int32_t nrb, ncb;         /* row blocks, column blocks */
  int64_t ntiles, nzc, nnz; /* nrb * ncb, non-empty (tile, column) pairs, entries */
  const int64_t* tdir_jc;
  const int64_t* tdir_ir;
  const uint16_t* jc;
  const uint32_t* cp;
  const uint16_t* ir;
} bfs_tile_info;
BFS_API int bfs_graph_tiles(bfs_graph* g, int32_t rb_bits, int32_t cb_bits, bfs_tile_info* info, void* stream);

/*
 * One SpMSV step with sorted output (Sec. 4.2, the multiway-merge way of
 * forming the union of the columns A(:, u) that the frontier selects):
 * t = A (x) f over the (select2nd, max) semiring of Sec. 3.2, masked by
 * not(visited) (Algorithm 3's t <- t (.) not(pi)), with every frontier value
 * the vertex's own id, so t(v) is the largest frontier vertex u with an arc
 * u -> v (an edge when undirected).  The merge is a stable radix sort of one
 * 64-bit key per selected entry; t comes out with ascending indices.
 *   frontier: device int32[nf] vertex ids (any order; repeats allowed);
 *   visited:  device bitmap uint32[ceil(n / 32)], bit v of word v / 32 set =
 *             v excluded from t; NULL = no mask;
 *   out_idx, out_val: device int32 arrays of capacity n (t's indices,
 *             ascending, and their values);
 *   *out_count (host): the number of entries of t.
 * Allocates temporary device memory of about 28 bytes per selected entry and
 * synchronises the stream.  Errors: BFS_ERR_INVALID_ARG (NULL pointers,
 * nf < 0, a frontier id outside [0, n)); BFS_ERR_INVALID_GRAPH (an adjacency
 * id outside [0, n)); BFS_ERR_OOM; BFS_ERR_CUDA.
 */
BFS_API int bfs_spmsv_sorted(bfs_graph* g, const int32_t* frontier, int32_t nf, const uint32_t* visited,
                             int32_t* out_idx, int32_t* out_val, int32_t* out_count, void* stream);

/*
 * Algorithm 3 with a single process, every level one bfs_spmsv_sorted step:
 * f <- {s}; while f is not empty: t <- A (x) f masked by not(pi); pi <- pi + t;
 * f <- t (in ascending id order).  Levels and parents are those of bfs_run;
 * the traversal takes a few kernels and a host read of t's size per level, so
 * it is a reference form of the sorted-output SpMSV, far slower than bfs_run.
 * parent_out, level_out: device int32[n].  Synchronises the stream.  Errors as
 * bfs_spmsv_sorted, and BFS_ERR_INVALID_ARG for a source outside [0, n).
 */
BFS_API int bfs_run_sorted(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out, void* stream);

/*
 * Symmetric half storage (the paper's closing note: an undirected graph's
 * adjacency is symmetric, so one triangle holds it): U keeps, of each row v,
 * the entries w > v, ascending.  bfs_graph_half builds U on the device the
 * first time (half the entries of a loop-free symmetric CSR) and keeps it with
 * g; the pointers stay valid until g is destroyed:
 *   offsets (int64[n + 1]), adj (int32[nnz]) on the device.
 * Synchronises the stream.  Errors: BFS_ERR_INVALID_ARG (NULL g or info),
 * BFS_ERR_UNSUPPORTED (a directed graph), BFS_ERR_OOM, BFS_ERR_CUDA.
 */
typedef struct bfs_half_info {
  int64_t nnz;
  const int64_t* offsets;
  const int32_t* adj;
} bfs_half_info;
BFS_API int bfs_graph_half(bfs_graph* g, bfs_half_info* info, void* stream);

/*
 * BFS that reads only U: a level pulls each unvisited v's U row from the top
 * (the first frontier entry is v's largest frontier neighbour above v, hence
 * its parent), then pushes each frontier vertex u to the entries of its U row
 * that are still unreached (atomicMax: the largest neighbour below them).
 * Levels and parents are those of bfs_run.  A few kernels and a host read per
 * level; a reference form of half storage, slower than bfs_run.
 * parent_out, level_out: device int32[n].  Builds U if g has none;
 * synchronises the stream.  The graph's ids are taken as valid, as in bfs_run
 * (BFS_VALIDATE at creation checks them).  Errors as bfs_graph_half, and
 * BFS_ERR_INVALID_ARG for a source outside [0, n) or NULL outputs.
 */
BFS_API int bfs_run_half(bfs_graph* g, int32_t source, int32_t* parent_out, int32_t* level_out, void* stream);

/* Waits for the stream (and for the copies of asynchronous host outputs of
 * runs on it) and returns (and clears) the device status of the last run
 * enqueued on it for graph g. */
BFS_API int bfs_sync(bfs_graph* g, void* stream);

/* Tuning of a graph (copied in / out). */
BFS_API int bfs_set_tuning(bfs_graph* g, const bfs_tuning* t);
BFS_API int bfs_get_tuning(const bfs_graph* g, bfs_tuning* t);

/*
 * Times bfs_run over `nroots` host roots (ids) for a small grid of tuning
 * candidates (bin degrees, pull thread degree, chunk degree, heuristic alpha,
 * beta, small_frontier, narrow_edges and ctas_per_sm; coordinate descent, two
 * sweeps), then bfs_run_batch over the first 64 of them for the batched
 * top-down limit; keeps the fastest as the graph's tuning and copies it to
 * *best.
 * Synchronises the stream; results never change, only speed.
 */
BFS_API int bfs_autotune(bfs_graph* g, const int32_t* roots, int32_t nroots, bfs_tuning* best, void* stream);

/* ---------------- the per-level variant selector network ---------------- */
/*
 * Network 12 -> 64 -> 64 -> 4, ReLU, float32, parameters packed flat as
 * W1[12][64], b1[64], W2[64][64], b2[64], W3[64][4], b3[4] (5,252 floats).
 * Inputs are the level features listed with bfs_level_features; outputs are
 * predicted log2 level times in microseconds of the four variants
 * BFS_VARIANT_TD_THREAD .. BFS_VARIANT_PULL, and the selector takes the
 * argmin (BFS_VARIANT_TILED is chosen only by BFS_SELECT_FORCED or a
 * schedule).  (The paper's counterpart is its choice between two SpMSV
 * accumulators by concurrency, Sec. 4.2.)
 */
#define BFS_MLP_PARAMS 5252
#define BFS_MLP_IN 12
#define BFS_MLP_OUT 4

/* Forward pass: X float[B][12], Y float[B][4] (device). */
BFS_API int bfs_mlp_forward(const float* params, const float* X, int32_t B, float* Y, void* stream);

/* Mean squared error over B x 4 against T float[B][4] and its gradient
 * grad float[5252]; loss float[1] (all device).  Deterministic (fixed
 * reduction order). */
BFS_API int bfs_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t B, float* grad,
                      float* loss, void* stream);

/* One Adam step (bias-corrected, step t >= 1) on params, with moments m, v (device). */
BFS_API int bfs_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr,
                 float beta1, float beta2, float eps, void* stream);

/* Full-batch Adam training for `steps` steps on device data; params updated in
 * place; loss_history (device float[steps]) may be NULL. */
BFS_API int bfs_selector_train(float* params, const float* X, const float* T, int32_t B, int32_t steps,
                       float lr, float* loss_history, void* stream);

/*
 * Training samples for the selector network from traversals of graph g: for
 * every root (host array) the traversal runs `reps` times with each of the
 * network's four variants forced at every level, and for every level k one
 * row is written:
 * X[row][0..11] = the level's features (bfs_level_features) and
 * T[row][v] = log2 of the median time in microseconds of level k under
 * variant v (host float arrays of max_rows rows).  *rows_out receives the
 * number of rows written (rows beyond max_rows are dropped).  Levels and
 * parents do not depend on the variant, so every run sees the same level
 * sequence.  Synchronises the stream.
 */
BFS_API int bfs_selector_collect(bfs_graph* g, const int32_t* roots, int32_t nroots, int32_t reps, float* X, float* T,
                                 int32_t max_rows, int32_t* rows_out, void* stream);

/* Sets (params != NULL, host float[5252]) or clears (NULL) the network used by
 * BFS_SELECT_LEARNED in this process. */
BFS_API int bfs_selector_set_params(const float* params);

/* Loads / saves the network as a raw little-endian float32[5252] file. */
BFS_API int bfs_selector_load(const char* path);
BFS_API int bfs_selector_save(const char* path);

/*
 * The 12 selector inputs of a level, from integer level statistics (host):
 * log2 n / 32, log2 nnz / 32, log2(1 + k) / 10, log2(1 + |f|) / 32,
 * log2(1 + sum deg f) / 32, |f| / n, sum deg f / nnz, unvisited / n,
 * unvisited edges / nnz, and the fraction of f with degree <= 32, <= 1024 and
 * larger.  "Unvisited" means not in levels 0..k, exactly the
 * unvisited_count / unvisited_edges fields of bfs_level_stat.  In float32:
 * every count is converted to float once, a ratio a / b is a * (1.0f / b), a
 * division by 32 or 10 is a product with 0.03125f or 0.1f.  The device
 * computes the same expressions inside bfs_run (its log2f may differ from the
 * host's in the last place).
 */
BFS_API int bfs_level_features(int32_t n, int64_t nnz, int32_t k, int64_t frontier_count,
                       int64_t frontier_edges, int64_t unvisited_count, int64_t unvisited_edges,
                       const int64_t* bin_count, float* out12);

/* Message of the last failed call on this thread ("" if none). */
BFS_API const char* bfs_last_error(void);

/* Library version string. */
BFS_API const char* bfs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BFS_GB300_H */
