/*
 * bfs.h - C ABI of the GB300 breadth-first-search library (libbfs.so).
 *
 * The library computes BFS distances on an undirected graph stored as CSR
 * (every edge present in both directions), following "Performance-Driven
 * Optimization of Parallel Breadth-First Search" (Bhaskar, Kanakagiri, 2025):
 * level-synchronous BFS (Section 2, Listing 1) with hybrid top-down /
 * bottom-up traversal (Section 2, BFS-Hybrid, Listing 2), a visited bitmap
 * (Section 2, BFS-VisitedBitmap, Listing 3) and plain, non-atomic distance
 * stores (Section 2, BFS-NonAtomic).  The distance of a vertex is the number
 * of edges on a shortest path from the source, the unique value every one of
 * those variants computes.
 *
 * Conventions for every entry point:
 *  - Return value: BFS_OK (0) or a negative BFS_E* code; bfs_strerror()
 *    names it.  No C++ exception crosses this boundary.
 *  - Vertex ids are int32 in [0, n); n < 2^31.
 *  - Unreachable vertices get distance -1 (int32 output) or 255 (uint8
 *    output); the paper's MAX_DISTANCE sentinel (Listing 1) maps to these.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is ordered on that stream.
 *  - Device pointers are plain CUDA device addresses (e.g. a torch tensor's
 *    data_ptr()) on the current device; host pointers are ordinary process
 *    memory (pinned memory makes copies faster but is not required).
 *  - The library owns what it allocates (graphs, workspaces, servers) until
 *    the matching *_free / *_destroy call; the caller owns every buffer it
 *    passes in.
 */
#ifndef GB300_BFS_H
#define GB300_BFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define BFS_OK 0
#define BFS_EINVAL (-1)   /* bad argument: null pointer, n out of range, bad CSR, src outside [0,n), k <= 0 */
#define BFS_ENOMEM (-2)   /* device or host allocation failed, or a memory budget is exceeded */
#define BFS_ECUDA (-3)    /* a CUDA runtime call failed (the CUDA error is logged to stderr) */
#define BFS_ETIMEOUT (-4) /* a bounded device-side wait (grid barrier) reached its time limit */
#define BFS_EAGAIN (-5)   /* a queue is full; retry later */
#define BFS_ERANGE (-6)   /* a distance does not fit the requested output type (uint8: > 254) */
#define BFS_ENOTFOUND (-7) /* unknown ticket or graph id */

/* ---- bfs_graph_upload flags ---- */
#define BFS_HOST_PTRS 0        /* row_ptr / col_idx are host pointers (copied to the device) */
#define BFS_DEVICE_PTRS 1      /* row_ptr / col_idx are device pointers (copied device-to-device) */
#define BFS_VALIDATE 2         /* check row_ptr[0]==0, monotone row_ptr, row_ptr[n]==m, 0<=col<n */
#define BFS_VALIDATE_SYMMETRY 4 /* also check that every arc (u,v) has its reverse (v,u) */
#define BFS_DEGREE_ORDER 8     /* store each adjacency list highest-degree neighbour first (ties by
                                  id); distances are unchanged, bottom-up scans stop sooner.
                                  Needs m < 2^31 and temporary device memory of 16*m bytes. */
#define BFS_NO_HEAD 16         /* do not build the per-vertex head table.  By default (when m < 2^31)
                                  the upload stores, for every vertex, its first two neighbours, the
                                  start of its list and its degree (16 bytes per vertex, after any
                                  degree ordering), so that a bottom-up probe of the first neighbours
                                  and a top-down degree lookup read one record instead of row_ptr and
                                  col_idx.  Distances are unchanged either way. */

/* ---- direction policies (bfs_params.policy) ----
 * Every policy yields the same distances; they differ only in work.
 * Level 0 is always top-down (Listing 2 starts with is_top_down = true). */
#define BFS_POLICY_AUTO 0     /* graph class rule of Section 3: average degree m/n below
                                 bfs_params.large_diameter_degree (7) -> top-down only, as
                                 BFS_POLICY_LOCAL when no vertex has more than 4096 entries (a
                                 longer list would be scanned by one warp there) and the launch is
                                 not BFS_LAUNCH_PER_LEVEL, as BFS_POLICY_TD_ONLY otherwise; else
                                 BFS_POLICY_EDGES */
#define BFS_POLICY_FRONTIER 1 /* the paper's BFS-Hybrid rule (Section 2, Listing 2): next level
                                 is top-down iff tau_inv*|F| < n (the paper's 5%: tau_inv = 20) */
#define BFS_POLICY_EDGES 2    /* the edge-count rule the paper cites as BFS-Hybrid-dagger
                                 (Section 2): top-down -> bottom-up when alpha*m_f > m_u;
                                 bottom-up -> top-down when beta*|F| < n and |F| shrank */
#define BFS_POLICY_TD_ONLY 3  /* top-down every level (the paper's large-diameter path, Section 3) */
#define BFS_POLICY_BU_FROM_1 4 /* top-down at level 0, bottom-up afterwards (testing) */
#define BFS_POLICY_SCRIPT 5   /* level L is bottom-up iff bit min(L,63) of bfs_params.script is set
                                 (bit 0 is ignored: level 0 is top-down); testing */
#define BFS_POLICY_LOCAL 6    /* top-down with several levels per grid barrier (Section 2, "Other
                                 Optimizations" (c): threads advance their own part of the frontier
                                 for several levels without merging; for Section 3's large-diameter
                                 graphs).  Each block expands its share of the frontier for up to
                                 bfs_params.local_levels levels on a shared-memory queue, distances
                                 are relaxed with atomicMin (a vertex reached first along a longer
                                 path is corrected and expanded again) and the search stops at the
                                 fixpoint, so the distances are the same exact values.  Runs as one
                                 persistent launch (BFS_LAUNCH_GRAPH runs it the same way; with
                                 BFS_LAUNCH_PER_LEVEL it is BFS_EINVAL); it always runs on the graph
                                 as uploaded (bfs_params.relabel is ignored).  Level records
                                 (bfs_single_ex) then describe super-steps: direction 2, frontier =
                                 global queue entries at its start, found = entries queued for the
                                 next, edges = entries examined (with stats), ns = device time. */

/* ---- launch modes (bfs_params.launch) ---- */
#define BFS_LAUNCH_PERSISTENT 0 /* one cooperative launch runs every level, grid barrier between levels */
#define BFS_LAUNCH_PER_LEVEL 1  /* one launch per phase; the host reads the frontier size each level */
#define BFS_LAUNCH_GRAPH 2      /* the persistent launch replayed from a captured CUDA graph */

typedef struct bfs_graph bfs_graph; /* opaque; owned by the library */

/* Tunable parameters.  bfs_params_default() fills the defaults; a zero field
 * keeps the default where noted. */
typedef struct bfs_params {
    int32_t policy;          /* BFS_POLICY_* (default BFS_POLICY_AUTO) */
    int32_t launch;          /* BFS_LAUNCH_* (default BFS_LAUNCH_PERSISTENT) */
    int32_t alpha;           /* BFS_POLICY_EDGES alpha (default 14) */
    int32_t beta;            /* BFS_POLICY_EDGES beta (default 24) */
    int32_t tau_inv;         /* BFS_POLICY_FRONTIER: top-down iff tau_inv*|F| < n (default 20) */
    int32_t large_diameter_degree; /* BFS_POLICY_AUTO threshold on m/n (default 7) */
    int32_t small_max;       /* top-down: vertices with degree < small_max (<= 32) are expanded
                                32 at a time by one warp; larger ones get a warp each (default 32) */
    int32_t chunk;           /* top-down: a vertex's adjacency is split into work items of at most
                                `chunk` edges (256..65535, default 256) */
    int32_t bu_warp_min;     /* bottom-up: an unvisited vertex with degree > bu_warp_min (<= 2^24) is
                                scanned on its own by the whole warp; smaller ones share the warp's
                                32-entry steps with their neighbours in the bitmap word (default 32) */
    int32_t threads_per_block; /* 128..1024, multiple of 32 (default 512) */
    int32_t blocks_per_sm;   /* 0 = as many as fit (cooperative launch limit) */
    int32_t timeout_ms;      /* limit of every device-side barrier wait (default 10000) */
    uint64_t script;         /* BFS_POLICY_SCRIPT direction bits */
    int32_t test_barrier_extra; /* testing only: grid barriers wait for this many blocks more than
                                   were launched, so a wait runs out and BFS_ETIMEOUT is returned */
    int32_t bu_chunk;        /* bottom-up: groups of 32 bitmap words a warp takes per grab from a shared
                                cursor (0 = static interleaved assignment, default; levels with fewer
                                unvisited vertices than bitmap words are always static) */
    int32_t bu_thread_max;   /* bottom-up: a vertex whose parent is not among its first entries (the
                                two of the head table, else the first aligned four) keeps scanning on
                                its own lane for up to this many more entries before the warp takes
                                over (default 32) */
    int32_t ms_lanes;        /* bfs_multi: sources per group (1..256, default 256) */
    int32_t ms_ring;         /* bfs_multi: frontier levels kept before they are written out (2..16,
                                default 16) */
    int32_t ms_heavy_min;    /* bfs_multi pull levels: vertices with more entries are scanned by a
                                whole warp (default 256) */
    int32_t ms_degree_order; /* bfs_multi pull levels visit vertices by decreasing degree (1, default)
                                or by id (0); used with ms_relabel = 0 (the renumbered copy is in
                                degree order already) */
    int32_t ms_alpha;        /* bfs_multi: a push level is followed by a pull level when
                                ms_alpha * (degree sum of the new frontier) > entries of vertices not
                                yet reached by every lane (default 2: a pull level scans those lists
                                nearly in full while lanes remain, unlike a single-source bottom-up
                                level, so it needs a denser frontier than alpha asks for) */
    int32_t ms_relabel;      /* bfs_multi: run on a copy of the graph whose vertices are renumbered by
                                decreasing degree (1, default; built once per graph on first use and
                                kept until bfs_graph_free: 4m + 8n bytes plus the row pointers), so the
                                masks most lists point to share cache lines; 0 = the graph as uploaded */
    int32_t relabel;         /* bfs_single: run on the same degree-renumbered copy (1; its head table,
                                visited mask and a host copy of the id map, 4n bytes, are added on
                                first use) so the frontier bits of high-degree vertices share cache
                                lines; distances are still written in the caller's ids.  0 (default):
                                the graph as uploaded */
    int32_t local_levels;    /* BFS_POLICY_LOCAL: levels a block advances on its own between two grid
                                barriers (1..4096, default 16) */
    int32_t local_threads;   /* BFS_POLICY_LOCAL: threads per block (64..512, multiple of 32, default
                                64; small blocks take small shares of the frontier, so the levels a
                                block runs alone are short) */
    int32_t serve_queue;     /* bfs_serve_*: queries submitted and not yet admitted before
                                bfs_serve_submit returns BFS_EAGAIN (0 = default 2^20) */
    int32_t reserved[1];
} bfs_params;

/* Per-query work counters (exact, deterministic: the frontier sets are unique
 * and the bottom-up scan stops at the first frontier neighbour in CSR order).
 * Edge counts are directed CSR entries. */
typedef struct bfs_stats {
    int32_t levels;          /* levels processed (eccentricity of src + 1) */
    int32_t td_levels;       /* of which top-down */
    int32_t bu_levels;       /* of which bottom-up */
    int32_t conversions;     /* queue <-> bitmap conversions (direction changes) */
    int64_t reached;         /* vertices with dist >= 0 */
    int64_t edges_reached;   /* sum of degrees over reached vertices (TEPS numerator x 2) */
    int64_t td_frontier;     /* sum over top-down levels of |F_L| */
    int64_t td_edges;        /* sum over top-down levels of the degrees in F_L */
    int64_t bu_unvisited;    /* sum over bottom-up levels of unvisited vertices of degree > 0 */
    int64_t bu_edges;        /* sum over bottom-up levels of entries examined (to the first hit) */
    int64_t bu_found;        /* sum over bottom-up levels of |F_{L+1}| */
    int64_t conv_frontier;   /* sum over conversions of |F| */
    int64_t supersteps;      /* BFS_POLICY_LOCAL: grid-synchronised super-steps (0 otherwise) */
    int64_t improved;        /* BFS_POLICY_LOCAL: successful relaxations (labels lowered), the source
                                excluded; above reached - 1 when a vertex was first reached along a
                                longer path (td_frontier: entries expanded, td_edges: examined) */
    int64_t init_ns;         /* persistent level-synchronous launch: device time from kernel entry to
                                the end of the per-query init (the counting variant's clock) */
    int64_t finish_ns;       /* ... and from the end of the last level to the end of the final
                                level-byte -> int32 expansion (0 where there is none) */
} bfs_stats;

/* One level's counters (optional detail). direction: 0 top-down, 1 bottom-up. */
typedef struct bfs_level_stat {
    int32_t direction;
    int32_t converted;       /* 1 if this level's frontier was converted before it ran */
    int64_t frontier;        /* |F_L| */
    int64_t edges;           /* top-down: degrees in F_L; bottom-up: entries examined */
    int64_t unvisited;       /* bottom-up: unvisited vertices of degree > 0 (0 for top-down) */
    int64_t found;           /* |F_{L+1}| */
    int64_t ns;              /* persistent launch: device time from the end of the previous level
                                (including any conversion) to the end of this one */
} bfs_level_stat;

/* Counters of one bfs_multi call (summed over its groups). */
typedef struct bfs_multi_stats {
    int32_t levels;          /* most levels of any group (largest eccentricity + 1) */
    int32_t push_levels;     /* levels run in push (top-down) form, summed over groups */
    int32_t pull_levels;     /* levels run in pull (bottom-up) form, summed over groups */
    int32_t groups;          /* source groups of up to ms_lanes sources */
    int64_t pushed_edges;    /* entries read by push levels */
    int64_t pulled_edges;    /* entries read by pull levels */
    int64_t output_bytes;    /* bytes written to dist (every output row counted per window) */
    int64_t pull_active;     /* sum over pull levels of vertices still missing an active lane (the
                                vertices whose lists a pull level reads) */
    int64_t push_frontier;   /* sum over push levels of frontier vertices (whose lists are pushed) */
    int64_t found;           /* sum over levels of vertices that gained at least one lane */
    int64_t reserved[1];
} bfs_multi_stats;

/* Per-level counts of bfs_single_nonatomic (level L expands the frontier F_L). */
typedef struct bfs_dup_level {
    int64_t frontier;        /* entries appended when F_L was found, duplicates included */
    int64_t unique;          /* distinct vertices among them (|F_L|) */
    int64_t edges;           /* list entries read expanding F_L */
} bfs_dup_level;

/* Totals of bfs_single_nonatomic. */
typedef struct bfs_dup_stats {
    int32_t levels;          /* levels expanded (eccentricity of src + 1) */
    int32_t pad;
    int64_t frontier_entries;/* sum over levels of appended entries, duplicates included */
    int64_t unique;          /* sum over levels of distinct frontier vertices (= reached vertices) */
    int64_t edges;           /* sum over levels of list entries read */
    int64_t reserved[4];
} bfs_dup_stats;

/* Message for a BFS_* code (static string). */
const char *bfs_strerror(int code);

/* Library version, major*10000 + minor*100 + patch. */
int bfs_version(void);

/*
 * Bounds-checked builds (compiled with -DGBFS_DEBUG_BOUNDS; the library's
 * stand-in for a device memory checker): every data-dependent global index of
 * the single-source kernels (level-synchronous and BFS_POLICY_LOCAL) is
 * checked against its array; the first out-of-range index is recorded and the
 * access is redirected to element 0, so the kernel completes.
 *  first_violation  0 if none, else bit 63 set | site << 48 | the low 48 bits
 *                   of the index (site numbers name the access in the source).
 *  checked          NULL or set to 1 when this library was built with the
 *                   checks (0: release build, first_violation is always 0).
 *  reset            nonzero clears the recorded violation.
 * Errors: BFS_EINVAL (null first_violation), BFS_ECUDA.
 */
int bfs_debug_bounds(uint64_t *first_violation, int *checked, int reset);

/* Fill *p with the defaults listed in bfs_params. */
void bfs_params_default(bfs_params *p);

/*
 * Copy a CSR graph to the current device (Section 2, Listing 1: rptr/col).
 *  row_ptr      n+1 offsets, int32 (row_ptr_bits = 32) or int64 (64); the
 *               device copy keeps this width.
 *  col_idx      m int32 neighbour ids.
 *  flags        BFS_HOST_PTRS or BFS_DEVICE_PTRS, optionally | BFS_VALIDATE
 *               (| BFS_VALIDATE_SYMMETRY).
 *  out          receives the graph handle.
 * The graph must be symmetric: the bottom-up phase (Listing 2) reads a
 * vertex's adjacency as its in-neighbours.  Self-loops and repeated entries
 * are allowed and do not change any distance.
 * Errors: BFS_EINVAL (null pointers, n < 1, n >= 2^31, m < 0, m >= 2^39, int32
 * offsets with m >= 2^31, a degree >= 2^31 - 2^16, failed validation),
 * BFS_ENOMEM, BFS_ECUDA.  Synchronous.
 */
int bfs_graph_upload(const void *row_ptr, int row_ptr_bits, const int32_t *col_idx, int64_t n,
                     int64_t m, int flags, bfs_graph **out);

/* Release a graph and its workspaces (NULL is ignored).  Synchronizes the device. */
void bfs_graph_free(bfs_graph *g);

/* Graph facts: vertex and entry counts, maximum degree, vertices of degree 0.
 * Any output pointer may be NULL. */
int bfs_graph_info(const bfs_graph *g, int64_t *n, int64_t *m, int64_t *max_degree,
                   int64_t *isolated);

/*
 * Single-source BFS distances (Section 2: BFS-Hybrid with BFS-VisitedBitmap
 * and non-atomic distance stores), default parameters.
 *  src    source vertex in [0, n).
 *  dist   int32[n], device or host memory (detected).  Device output is
 *         written in stream order; pinned (page-locked) host output is
 *         written by the kernel directly through its device alias (except
 *         under BFS_POLICY_LOCAL, whose atomic relaxations stay on the
 *         device); other host output is staged on the device and copied back
 *         before return.
 * Blocks until the query has finished (the device status word is read back).
 * Queries on one graph are serialized on the device (they share its workspace).
 * Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA, BFS_ETIMEOUT.
 */
int bfs_single(bfs_graph *g, int32_t src, int32_t *dist, void *stream);

/*
 * bfs_single with explicit parameters and optional counters.
 *  params       NULL = defaults.
 *  stats        NULL, or receives the query's totals.
 *  levels       NULL, or an array of level_cap entries receiving per-level
 *               records for levels 0..min(levels, level_cap)-1: direction,
 *               converted, frontier, found and (persistent launch) ns always;
 *               edges and unvisited only when stats is non-NULL (the counting
 *               variant of the kernel runs only then).  Unused entries stay zero.
 */
int bfs_single_ex(bfs_graph *g, int32_t src, int32_t *dist, const bfs_params *params,
                  bfs_stats *stats, bfs_level_stat *levels, int32_t level_cap, void *stream);

/*
 * Enqueue one single-source query (as bfs_single_ex without statistics) and
 * return without waiting for it, so that a caller with many queries keeps the
 * device busy: the next query's launch is queued while this one runs.
 *  dist   int32[n] device memory, or pinned host memory written through its
 *         device alias (not under BFS_POLICY_LOCAL); owned by the caller and
 *         written when the stream reaches the query.  Pageable host memory:
 *         BFS_EINVAL (it would need a staged copy and a wait).
 * Queries on one graph run in submission order on the device, whichever streams
 * they name (they share its workspace), and each dist buffer is complete once
 * its stream passes the query.  A query's device status (BFS_ETIMEOUT) is kept
 * on the device until bfs_single_wait reports it.
 * Returns BFS_OK once enqueued; BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA.
 */
int bfs_single_async(bfs_graph *g, int32_t src, int32_t *dist, const bfs_params *params, void *stream);

/*
 * Wait until every single-source query enqueued on g has finished and return
 * the first failed status (BFS_ETIMEOUT) among the queries since the previous
 * wait (a failure already returned by a synchronous call is not repeated), or
 * BFS_OK; the recorded status is then cleared.  BFS_OK at once if g has had no
 * single-source query.  Errors: BFS_EINVAL (g NULL), BFS_ECUDA.
 */
int bfs_single_wait(bfs_graph *g);

/*
 * Distances from k sources at once (multi-source BFS: the level-synchronous
 * loop of Section 2 run for up to 256 sources together, one bit per source in
 * per-vertex masks; sparse levels push as in Listing 1, dense levels pull as in
 * Listing 2's bottom-up scan).
 *  srcs       host int32[k], each in [0, n); repeats allowed.
 *  dist       [k][n] row-major (row i = distances from srcs[i]), device or host
 *             memory (detected); dist_bits 8 (uint8, 255 = unreachable) or 32
 *             (int32, -1 = unreachable).
 * Sources are processed in groups of bfs_params.ms_lanes (default 256).  The
 * first call on a graph builds its degree-renumbered copy (bfs_params.ms_relabel)
 * and the group workspace: (2 + ms_ring) * 32 bytes per vertex for 256 lanes.
 * Blocks until done.  Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA, BFS_ERANGE
 * (uint8 output and a distance above 254: dist is then incomplete).
 */
int bfs_multi(bfs_graph *g, const int32_t *srcs, int32_t k, void *dist, int dist_bits, void *stream);

/* bfs_multi with parameters (NULL = defaults) and optional counters (NULL = none). */
int bfs_multi_ex(bfs_graph *g, const int32_t *srcs, int32_t k, void *dist, int dist_bits,
                 const bfs_params *params, bfs_multi_stats *stats, void *stream);

/*
 * A BFS tree from finished distances (Graph500-style parent array; the paper
 * computes distances only).  dist: device int32[n] from a query on g (any
 * entry point); parent: device int32[n], written on `stream`: the parent of a
 * reached vertex v other than the source is the first vertex u of v's list (in
 * the library's list order, see BFS_DEGREE_ORDER) with dist[u] = dist[v] - 1;
 * the vertex at distance 0 is its own parent; unreached vertices get -1.
 * A reached vertex with no such neighbour (dist not a BFS result of g) gets -1.
 * Asynchronous.  Calls on one graph share a small device workspace; the
 * library orders them on the device (each call waits for the previous one's
 * completion, whatever stream either used), so calls from several streams or
 * threads are safe but do not overlap.  Errors: BFS_EINVAL (null or host
 * pointers), BFS_ECUDA.
 */
int bfs_parents(bfs_graph *g, const int32_t *dist, int32_t *parent, void *stream);

/*
 * The paper's BFS-NonAtomic top-down traversal (Section 2, Listing 1 with the
 * byte-map visited set of Listing 3), kept to measure its duplicates: a thread
 * that finds neighbour v unvisited marks it (visited byte, dist = L + 1) with
 * plain stores and appends it to the next frontier without claiming it, so two
 * threads that test v at the same time both append it.  Distances are exact
 * (every writer of a level stores the same value).  On a GPU a level's tests
 * run nearly at once and duplicates would multiply from level to level if they
 * were expanded again, so before a level is expanded its entries are reduced
 * to distinct vertices without atomics (each entry stores its index into a
 * per-vertex slot; the entry whose index remains is kept).
 * Top-down levels only, one launch sequence per level, blocks until done.
 *  dist       device int32[n] (-1 = unreachable), written on `stream`.
 *  stats      NULL or totals; levels NULL or per-level counts for the first
 *             level_cap levels.
 * The first call allocates its workspace (5 bytes per vertex and two queues of
 * n + m + 1 entries, kept until bfs_graph_free).  Errors: BFS_EINVAL (also
 * n + m + 1 >= 2^31), BFS_ENOMEM, BFS_ECUDA.
 */
int bfs_single_nonatomic(bfs_graph *g, int32_t src, int32_t *dist, bfs_dup_stats *stats, bfs_dup_level *levels,
                         int32_t level_cap, void *stream);

/* bfs_single_nonatomic's treatment of duplicate frontier entries. */
#define BFS_DUP_DEDUP 0   /* reduce each level's appended entries to distinct vertices (without atomics)
                             before expanding them (bfs_single_nonatomic) */
#define BFS_DUP_EXPAND 1  /* expand every appended entry, duplicates included, as the paper's variant does
                             (Section 2: duplicates are processed again at the next level); a level's
                             entries then also count the copies, and when they outgrow the queues
                             (n + m + 1 entries) or the long-list records the call returns BFS_ENOMEM
                             without writing past them */

/* bfs_single_nonatomic with the duplicate mode (BFS_DUP_DEDUP or BFS_DUP_EXPAND).  Per level,
 * levels[L].frontier counts the entries expanded at level L in BFS_DUP_EXPAND mode (the appended
 * entries), levels[L].unique the distinct vertices among them, levels[L].edges the list entries read
 * (every copy of a vertex reads its list again). */
int bfs_single_nonatomic_ex(bfs_graph *g, int32_t src, int32_t *dist, int mode, bfs_dup_stats *stats,
                            bfs_dup_level *levels, int32_t level_cap, void *stream);

/* ---- autotuner ---- */

/* Outcome of bfs_tune. */
typedef struct bfs_tune_report {
    int32_t trials;          /* parameter settings timed */
    int32_t sources;         /* sample sources per trial */
    double start_ms;         /* median BFS time with the starting parameters */
    double best_ms;          /* median BFS time with the returned parameters */
    int64_t reserved[4];
} bfs_tune_report;

/*
 * Pick single-source parameters for graph g by coordinate descent, one field
 * at a time (two sweeps).  Small-world graphs (average degree >= 7): policy
 * (Section 2's frontier rule or the edge-count rule), alpha, beta, tau_inv,
 * relabel, chunk, small_max, bu_thread_max, bu_warp_min, bu_chunk,
 * threads_per_block, blocks_per_sm.  Section 3's large-diameter class:
 * policy (top-down level-synchronous or BFS_POLICY_LOCAL), local_levels,
 * local_threads, chunk, threads_per_block, blocks_per_sm.  A setting's time is
 * the mean over the k sample sources of each source's best of three timed
 * runs (CUDA events, after a warm-up run); it is kept when at least 2% faster.
 * Every setting's distances must hash identically to the starting setting's;
 * a mismatch aborts with BFS_ECUDA.  base = NULL starts from the defaults.
 * Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA, BFS_ETIMEOUT.
 */
int bfs_tune(bfs_graph *g, const int32_t *srcs, int32_t k, const bfs_params *base, bfs_params *out,
             bfs_tune_report *report);

/*
 * Pick bfs_multi (and serving-group) parameters for graph g: ms_alpha (the
 * push -> pull switch), ms_heavy_min, ms_ring, ms_lanes, ms_relabel and
 * ms_degree_order, by the same coordinate descent; a setting's time is the
 * best of three timed bfs_multi calls on all k sources (dist_bits 8 or 32),
 * whose whole output must hash identically across settings.  Needs k*n*
 * dist_bits/8 bytes of device memory for the output.
 * Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA, BFS_ERANGE.
 */
int bfs_tune_multi(bfs_graph *g, const int32_t *srcs, int32_t k, int dist_bits, const bfs_params *base,
                   bfs_params *out, bfs_tune_report *report);

typedef struct bfs_graphset bfs_graphset;

/*
 * Pick graph-set parameters (threads_per_block <= 512, blocks_per_sm, alpha,
 * beta of the block-local direction rule) for one bfs_graphset_run over set s
 * from srcs (one local source per graph); a setting's time is the best of
 * three timed runs, whose distances must hash identically across settings.
 * Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA.
 */
int bfs_tune_graphset(bfs_graphset *s, const int32_t *srcs, const bfs_params *base, bfs_params *out,
                      bfs_tune_report *report);

/* ---- graph sets: many small graphs, one source each, one launch ---- */

/* bfs_graphset (declared above) is opaque and owned by the library. */

/* Counters of one bfs_graphset_run. */
typedef struct bfs_graphset_stats {
    int32_t graphs;          /* graphs in the set */
    int32_t max_levels;      /* largest eccentricity + 1 */
    int32_t blocks;          /* persistent blocks launched */
    int32_t pad;
    int64_t levels;          /* levels processed, summed over graphs */
    int64_t td_levels;       /* of which top-down */
    int64_t bu_levels;       /* of which bottom-up */
    int64_t reserved[4];
} bfs_graphset_stats;

/*
 * Upload a set of `count` independent CSR graphs (host pointers), each with
 * local vertex ids 0..n_i-1:
 *  voff     int64[count+1]: graph i owns global vertex slots voff[i]..voff[i+1]-1
 *           (n_i = voff[i+1] - voff[i] >= 1, n_i <= 2^19).
 *  eoff     int64[count+1]: graph i's neighbour ids are col[eoff[i]..eoff[i+1]).
 *  row_ptr  int64[voff[count] + count]: graph i's n_i+1 local row pointers start
 *           at row_ptr[voff[i] + i] (each starts at 0).
 *  col      int32[eoff[count]] local neighbour ids.
 *  flags    BFS_VALIDATE checks every graph's CSR on the host.
 * Every graph must be symmetric.  Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA.
 */
int bfs_graphset_upload(const int64_t *voff, const int64_t *eoff, const int64_t *row_ptr,
                        const int32_t *col, int32_t count, int flags, bfs_graphset **out);

/* Release a graph set (NULL is ignored). */
void bfs_graphset_free(bfs_graphset *s);

/*
 * BFS of every graph of the set from its own source in ONE persistent launch
 * (Section 2's hybrid BFS per graph, run inside one block with shared-memory
 * bitmaps; blocks take graphs largest first).
 *  srcs    host int32[count], local source id of each graph.
 *  dist    int32[voff[count]] (device or host, detected): graph i's distances
 *          at dist[voff[i] .. voff[i+1]), -1 = unreachable.
 *  params  NULL = defaults (uses alpha, beta, threads_per_block <= 512,
 *          blocks_per_sm).
 *  stats   NULL or receives counters.
 * Blocks until done.  Errors: BFS_EINVAL, BFS_ENOMEM, BFS_ECUDA.
 */
int bfs_graphset_run(bfs_graphset *s, const int32_t *srcs, int32_t *dist, const bfs_params *params,
                     bfs_graphset_stats *stats, void *stream);

/* ---- serving: resident graphs, a stream of queries, continuous batching ---- */

typedef struct bfs_server bfs_server; /* opaque; owned by the library */

/* Timeline of one query (steady-clock nanoseconds). */
typedef struct bfs_query_stats {
    int64_t submit_ns;       /* bfs_serve_submit returned */
    int64_t start_ns;        /* admitted into a lane */
    int64_t done_ns;         /* result complete in the caller's buffer */
    int32_t levels;          /* levels the query ran (its eccentricity + 1) */
    int32_t lane;            /* lane it ran in */
    int32_t graph_id;
    int32_t status;          /* BFS_OK or an error code */
    int64_t reserved[2];
} bfs_query_stats;

/*
 * Start a server on the current device.  The server runs the queries
 * of each registered graph in one 64-lane multi-source group (Section 2's
 * level-synchronous loop for all lanes at once); a query waiting for a lane
 * joins the running group at its next level and leaves when its frontier is
 * empty, so queries overlap on the device as they arrive (continuous
 * batching).  Admission is bounded by mem_budget bytes of device memory: a
 * graph's group state (about (8*(2+ms_ring) + 16) bytes per vertex) when its
 * first query arrives, and a 4n-byte staging buffer for every running query
 * whose output is host memory.  When a graph's queries cannot be admitted
 * because other groups hold the budget, those groups stop admitting, finish
 * their running queries and release their memory, so every graph is served
 * in turn even when the budget holds one group at a time; a query whose
 * group alone exceeds the budget completes with status BFS_ENOMEM.  A device
 * wait that runs out (BFS_ETIMEOUT) fails the running queries of that group
 * only (their status), the group is rebuilt for the next query, and the
 * server keeps serving; a CUDA error makes later calls return it.  Uses params->ms_ring, ms_heavy_min, tau_inv
 * (levels run push when tau_inv * |F| < n, else pull) and large_diameter_degree:
 * a graph with m < large_diameter_degree * n (Section 3's large-diameter class)
 * gets a high-priority stream, writes each distance as it is found, and runs
 * consecutive push levels in one persistent launch (bounded device waits of
 * params->timeout_ms each; params->test_barrier_extra as in bfs_params).
 * params->serve_queue bounds the submitted, not yet admitted queries.  Every
 * graph has its own worker thread.
 * NULL params = defaults.
 */
int bfs_serve_create(size_t mem_budget, const bfs_params *params, bfs_server **out);

/* Register a graph (it stays owned by the caller and must outlive the server). */
int bfs_serve_add_graph(bfs_server *srv, bfs_graph *g, int32_t *graph_id);

/*
 * Queue the query (graph_id, src).  dist_out: int32[n], device or host memory
 * (detected; pinned host memory avoids a synchronous copy), owned by the caller
 * and valid until the query is reported done.  The server writes it on its own
 * streams, which are not ordered with the caller's: device work that writes
 * the buffer must have completed before the call.  Returns a ticket.
 * Errors: BFS_EINVAL, BFS_ENOTFOUND (graph id), BFS_EAGAIN (queue full).
 */
int bfs_serve_submit(bfs_server *srv, int32_t graph_id, int32_t src, int32_t *dist_out, uint64_t *ticket);

/* *done = 1 once the query's distances are complete.  A completed ticket is
 * reported once (stats filled if non-NULL); later calls return BFS_ENOTFOUND. */
int bfs_serve_poll(bfs_server *srv, uint64_t ticket, int *done, bfs_query_stats *stats);

/* Block until the query completes (timeout_us < 0: no limit); then as poll.
 * Returns BFS_ETIMEOUT if the limit passes first (the query keeps running). */
int bfs_serve_wait(bfs_server *srv, uint64_t ticket, int64_t timeout_us, bfs_query_stats *stats);

/* Finish running queries, drop queued ones, stop the threads, free the server. */
void bfs_serve_destroy(bfs_server *srv);

/*
 * bfs_single distances without any memory allocation (the paper has no
 * counterpart; this is a library-usage variant).
 *
 * For callers that cannot allocate device memory when they run a query: code
 * confined to a memory pool or arena it does not own, contexts where an
 * allocation could block on the allocator or synchronize the device, or
 * processes that reserved all device memory in advance.  The caller passes
 * the graph and the output as device pointers; the kernel's scratch (bitmaps,
 * frontier queues, control block) lives in one static device array of
 * 64 MiB that the library reserves on every GPU where it is loaded, until the
 * process exits.  Nothing is allocated by this call: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *  row_ptr, row_ptr_bits, col_idx, n, m   the CSR graph as in
 *        bfs_graph_upload, but already in DEVICE memory and not copied or
 *        validated (it must be a valid symmetric CSR).  col_idx must start on
 *        a 16-byte boundary (the kernel reads it with aligned 16-byte loads,
 *        which may touch up to 3 entries past m inside the 16-byte block that
 *        holds the last entry; that block must be readable device memory, as
 *        it is for any cudaMalloc or caching-allocator buffer); row_ptr must
 *        be aligned to its width and dist to 4 bytes.  A misaligned pointer
 *        returns BFS_EINVAL before anything is launched.
 *  src   source vertex in [0, n).
 *  dist  device int32[n] output (-1 = unreachable).
 * Limit: the scratch needs about 24.5*n + m/15 bytes (each of its eleven
 * regions rounded up to 256 bytes); larger graphs get BFS_ENOMEM.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents: calls
 * that may overlap on the GPU (other streams, unordered host threads) race
 * with each other and must be serialized by the caller.
 * Uses the default parameters with the level-synchronous kernel (top-down
 * only below average degree 7, else the edge-count rule).  Blocks until the
 * query has finished.  Errors: BFS_EINVAL, BFS_ENOMEM (too large), BFS_ECUDA,
 * BFS_ETIMEOUT.
 */
int bfs_single_noalloc(const void *row_ptr, int row_ptr_bits, const int32_t *col_idx, int64_t n,
                       int64_t m, int32_t src, int32_t *dist, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_BFS_H */
