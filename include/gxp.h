/*
 * gxp.h — C-ABI of the GB300 GAS superstep engine (libgxp.so).
 *
 * The engine runs the per-superstep iteration of GX-Plug's daemon
 * (Section II-A1 and IV-A1: the algorithm template MSGGen / MSGMerge /
 * MSGApply) over graph partitions held on one GPU, with the paper's
 * synchronization caching and skipping between partitions (Section III-B,
 * Algorithm 3) and its pipeline shuffle for edge blocks streamed from host
 * memory (Section III-A, Algorithms 1-2, Lemma 1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns gxp_status; none aborts, throws or exits.
 *   gxp_status_string() names a code; gxp_last_error() gives the detail of
 *   the last failure on a context.
 * - Validation errors (GXP_E_INVAL, GXP_E_UNSUPPORTED, GXP_E_STATE) are
 *   returned synchronously and leave the context unchanged.
 * - Errors raised asynchronously on the GPU (a CUDA fault, a device-side
 *   bounds check, a device wait that ran out of time) are returned by the
 *   next call that synchronizes with the device. After GXP_E_CUDA,
 *   GXP_E_TIMEOUT, GXP_E_BOUNDS or GXP_E_LOST the context is poisoned: later
 *   calls return GXP_E_STATE until gxp_destroy().
 * - Pointers: unless a flag says otherwise, array arguments may be host or
 *   device pointers (the library copies through unified addressing). Input
 *   arrays are copied; the caller keeps ownership and may free them when the
 *   call returns. Output arrays are caller-allocated.
 * - Vertex ids are uint32 (at most 2^32 - 2 vertices: 0xFFFFFFFF is the
 *   "infinite" distance of SSSP); edge counts are uint64, at most 2^32 - 1
 *   edges per partition.
 * - One host thread at a time per context, except gxp_query_submit /
 *   gxp_query_poll, which are thread-safe.
 */
#ifndef GXP_H
#define GXP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GXP_API __attribute__((visibility("default")))

typedef enum gxp_status {
    GXP_OK = 0,
    GXP_E_INVAL = 1,        /* bad argument: null pointer, size, range, format */
    GXP_E_NOMEM = 2,        /* device or pinned host allocation failed, or over mem_budget */
    GXP_E_CUDA = 3,         /* a CUDA runtime call or kernel failed */
    GXP_E_TIMEOUT = 4,      /* a device-side wait exceeded timeout_ns */
    GXP_E_BOUNDS = 5,       /* a device-side bounds check found an out-of-range index */
    GXP_E_STATE = 6,        /* call out of order, or context poisoned by an earlier error */
    GXP_E_UNSUPPORTED = 7,  /* valid but not implemented combination */
    GXP_E_BUSY = 8,         /* no free query slot / queue full (serving) */
    GXP_E_LOST = 9          /* an exchange between partitions did not arrive: the superstep's
                               delivery mark was missing when its stats were read (the lazy
                               upload of Section III-B2 lost a message); poisons the context */
} gxp_status;

/* Host-side fault injection (gxp_config.fault, or the GXP_FAULT environment
 * variable "kind[:n][,kind[:n]...]" with kinds alloc, h2d, sync, timeout).
 * None makes the GPU fault, trap or hang: each fails one host-side event on
 * purpose so that the error paths can be tested.
 *  - ALLOC:     the fault_at-th device allocation of the context fails as an
 *               out-of-memory would: the call returns GXP_E_NOMEM and the
 *               context stays usable (the graph must be loaded again).
 *  - H2D:       the fault_at-th host-to-device copy is not enqueued: the call
 *               returns GXP_E_CUDA and the context is poisoned.
 *  - SYNC_DROP: the fault_at-th exchange between partitions is dropped (its
 *               kernels are not launched); the next read of the superstep
 *               statistics finds its delivery mark missing: GXP_E_LOST, and
 *               the context is poisoned.
 *  - TIMEOUT:   every bounded device-side wait gives up at once (it then
 *               waits for its own copies in flight): GXP_E_TIMEOUT. Only the
 *               kernel of gxp_superstep_min_noalloc waits on the device, and
 *               it reads the GXP_FAULT variable ("timeout") on every call. */
typedef enum gxp_fault {
    GXP_FAULT_NONE = 0,
    GXP_FAULT_ALLOC = 1,
    GXP_FAULT_H2D = 2,
    GXP_FAULT_SYNC_DROP = 3,
    GXP_FAULT_TIMEOUT = 4
} gxp_fault;

typedef enum gxp_algo {
    GXP_ALGO_SSSP = 0,      /* Bellman-Ford shortest paths (Section V-A) */
    GXP_ALGO_CC = 1,        /* min-label propagation = weakly connected components */
    GXP_ALGO_PAGERANK = 2,  /* PageRank with dangling-mass redistribution */
    GXP_ALGO_PPR = 3,       /* personalized PageRank from `source`: PageRank whose teleport and
                               dangling mass return to the source (r_0 = e_source) */
    GXP_ALGO_LP = 4         /* label propagation (Section V-A's LP): l_0[v] = v; each superstep a
                               vertex takes the label most of its in-edges carry, ties to the
                               smallest label; vertices without in-edges keep theirs. Synchronous
                               (Jacobi); it need not converge (the paper caps it at 15 supersteps:
                               pass max_steps = 15 to gxp_run) */
} gxp_algo;

/* The three template functions of Section IV-A1, as built-in operators. */
typedef enum gxp_msggen {
    GXP_GEN_RELAX = 0,      /* m = d[u] + w(u,v), saturating at 0xFFFFFFFE; none if d[u] = INF */
    GXP_GEN_LABEL = 1,      /* m = l[u] */
    GXP_GEN_CONTRIB = 2     /* m = r[u] / outdeg(u), fp32 */
} gxp_msggen;

typedef enum gxp_merge {
    GXP_MERGE_MIN = 0,      /* uint32 minimum, exact */
    GXP_MERGE_SUM = 1,      /* fp32 sum in a fixed order (deterministic) */
    GXP_MERGE_MODE = 2      /* the most frequent uint32 message, ties to the smallest, exact */
} gxp_merge;

typedef enum gxp_apply {
    GXP_APPLY_MIN = 0,      /* x' = min(x, m); changed if x' != x */
    GXP_APPLY_PAGERANK = 1, /* r' = (1-d)/N + d (m + D/N), D = dangling mass; personalized
                               PageRank: r' = d m, plus (1-d) + d D at the source */
    GXP_APPLY_SET = 2       /* x' = m if the vertex received messages, else x; changed if x' != x */
} gxp_apply;

typedef enum gxp_format {
    GXP_FMT_COO = 0,        /* idx0 = src[n_edges] (uint32 global), idx1 = dst[n_edges] (uint32 global) */
    GXP_FMT_CSC = 1,        /* idx0 = col_ptr[n_local + 1] (uint64, starts at 0), idx1 = src[n_edges] (uint32 global);
                               edges of local dst v are src[col_ptr[v] .. col_ptr[v+1]) */
    GXP_FMT_CSR = 2         /* idx0 = row_ptr[n_vertices + 1] (uint64) over global sources,
                               idx1 = dst[n_edges] (uint32 global, all inside the partition) */
} gxp_format;

typedef enum gxp_dtype { GXP_U32 = 0, GXP_F32 = 1, GXP_F64 = 2 } gxp_dtype;

typedef struct gxp_config {
    uint64_t mem_budget;        /* bytes of device memory the context may hold; 0 = no limit */
    uint32_t tile_items;        /* in-edges per hub part (a part of a high-in-degree vertex's
                                   in-edges reduced by one warp); 0 = 2048; <= 2^24 */
    uint32_t hub_items;         /* vertices with more in-edges than this are hubs, split into
                                   parts of tile_items edges; the rest are packed into
                                   32-row sliced-ELL slices; 0 = tile_items / 2; <= 2^24 */
    uint64_t timeout_ns;        /* limit for any device-side wait; 0 = 2e9 (2 s) */
    uint32_t check_bounds;      /* 1: kernels range-check every gathered index */
    uint32_t max_slots;         /* unused (serving takes gxp_serve_opts.max_slots); 0 */
    uint32_t pipeline_depth;    /* ring slots of the pipeline shuffle; 0 = 3 */
    uint32_t keep_ids;          /* 0: a single-partition graph is renumbered internally by
                                   decreasing in-degree, so the most gathered values share cache
                                   lines (values, sources and labels are mapped back: results
                                   are in input ids); 1: keep the input order */
    uint32_t direction;         /* gxp_direction of SSSP / CC supersteps: GXP_DIR_AUTO (0,
                                   default), GXP_DIR_PULL or GXP_DIR_PUSH. With several
                                   partitions a push relaxes, in each partition, the in-edges
                                   from its own changed vertices and from its cached copies of
                                   changed remote vertices (delivered by the exchange). */
    uint32_t push_div;          /* GXP_DIR_AUTO pushes a superstep when (frontier out-edges +
                                   frontier items) * push_div <= the graph's edges; 0 = 8 */
    uint32_t cache_slots;       /* synchronization caching (Section III-B2) with a budget: remote
                                   copies each partition keeps cached between supersteps.
                                   0 = all of them; GXP_CACHE_NONE = none. With a budget the cache
                                   is LRU-weighted (see gxp_cache_get): a copy enters when a
                                   superstep uses it, its weight decays by half per superstep and
                                   rises with its reads, the lowest weights are evicted. Cached
                                   copies are refreshed by the lazy upload of changed boundary
                                   vertices; a used copy that is not cached is downloaded from its
                                   owner (gxp_stats.cache_downloads). Values are the same either
                                   way. */
    uint32_t fault;             /* gxp_fault injected into this context; 0 = none (GXP_FAULT may
                                   still name one) */
    uint32_t fault_at;          /* which event of that kind fails, from 1; 0 = the first */
    uint32_t reserved[1];
} gxp_config;

#define GXP_CACHE_NONE 0xFFFFFFFFu

/* Direction of the min-label supersteps (SSSP, CC). Both give the same values
 * and the same changed sets after every superstep (Jacobi order):
 *  - PULL: every destination merges all of its in-edges (dst-sorted layout);
 *  - PUSH: only the out-edges of the vertices changed by the previous
 *    superstep (the frontier) are relaxed, into the next values with atomic
 *    min (src-sorted copy of the edges, built at the first gxp_begin that
 *    needs it: 4 bytes per vertex + 4 or 8 bytes per edge);
 *  - AUTO: per superstep on the device, push while the frontier's out-edges
 *    are a small share of all edges (push_div), else pull. A push needs the
 *    previous superstep's changed vertices as a list; with several
 *    partitions a pull superstep writes that list only when the frontier it
 *    read was within 4x the push limit, so a frontier that shrinks below the
 *    limit from above 4x it in one superstep is pulled once more. */
typedef enum gxp_direction {
    GXP_DIR_AUTO = 0,
    GXP_DIR_PULL = 1,
    GXP_DIR_PUSH = 2
} gxp_direction;

/* Fill *cfg with the defaults above (all zero = defaults). */
GXP_API void gxp_config_default(gxp_config* cfg);

typedef struct gxp_ctx gxp_ctx;

typedef struct gxp_stats {
    uint64_t supersteps;            /* supersteps run since the last gxp_begin */
    uint64_t edges_scanned;         /* edges read by supersteps since gxp_begin */
    uint64_t last_changed;          /* vertices changed by the last superstep */
    uint64_t last_boundary_changed; /* of which boundary vertices uploaded by its sync */
    uint64_t syncs_done;            /* exchanges performed (Algorithm 3) */
    uint64_t syncs_skipped;         /* exchanges skipped (Section III-B3) */
    uint64_t sync_pairs;            /* (id, value) pairs moved by all syncs */
    double   last_l1_delta;         /* PageRank: sum |r_{t+1} - r_t| of the last superstep */
    double   last_dangling;         /* PageRank: dangling mass D of the current ranks */
    double   last_superstep_ms;     /* device time of the last superstep incl. its sync */
    uint64_t device_bytes;          /* device memory held by the context */
    uint64_t push_supersteps;       /* of the supersteps, those run in push direction */
    uint64_t cache_downloads;       /* remote values downloaded because they were not cached
                                       (gxp_config.cache_slots), summed over supersteps */
    double   last_kernel_ms;        /* device time of the last superstep's compute kernel alone
                                       (MSGGen + MSGMerge + MSGApply, without its sync); gxp_run's
                                       device-driven loop: the average superstep */
    uint64_t persistent_launches;   /* gxp_run launches of the persistent superstep loop since
                                       gxp_begin (small single-partition SSSP / CC graphs: one
                                       cooperative kernel runs up to 32 supersteps) */
    uint64_t reserved[2];
} gxp_stats;

/* ------------------------------------------------------------ lifecycle -- */

/* Create a context on CUDA device `device` (Section IV-C: the device is
 * initialised once and reused by every later call). cfg may be NULL. */
GXP_API gxp_status gxp_init(int device, const gxp_config* cfg, gxp_ctx** out);

/* Release every resource of the context. NULL is a no-op. */
GXP_API void gxp_destroy(gxp_ctx* ctx);

GXP_API const char* gxp_status_string(gxp_status s);
GXP_API const char* gxp_last_error(const gxp_ctx* ctx);

/* Use `stream` (a cudaStream_t, or NULL for the context's own stream) for
 * all later device work of the context. */
GXP_API gxp_status gxp_set_stream(gxp_ctx* ctx, void* stream);

/* ---------------------------------------------------------------- graph -- */

/* Declare the graph: n_vertices in total, split into n_parts partitions that
 * own contiguous destination-id ranges [part_begin[p], part_begin[p+1])
 * (Section II-B: the upper system partitions the graph across nodes).
 * part_begin has n_parts + 1 entries, part_begin[0] = 0,
 * part_begin[n_parts] = n_vertices, non-decreasing; NULL = even split.
 * Drops any previously loaded graph. */
GXP_API gxp_status gxp_create_graph(gxp_ctx* ctx, uint64_t n_vertices, uint32_t n_parts,
                                    const uint64_t* part_begin);

/* Load the in-edges of partition `part` (every edge whose destination the
 * partition owns) in format `fmt` (see gxp_format), with optional uint32
 * weights (NULL = unweighted; weights are in the order of idx1 for CSC/CSR and
 * of the edge list for COO). The engine builds its dst-sorted edge blocks and
 * the vertex-edge mapping table from it (Section II-B: fixed-size edge blocks
 * paired with vertex blocks). Ownership of the arrays stays with the caller.
 * Errors: GXP_E_INVAL for an out-of-range id, a destination outside the
 * partition, a non-monotone offset array, or more than 2^32-1 edges. */
GXP_API gxp_status gxp_load_partition(gxp_ctx* ctx, uint32_t part, gxp_format fmt,
                                      uint64_t n_edges, const void* idx0, const uint32_t* idx1,
                                      const uint32_t* weights);

/* ------------------------------------------------------- vertex values -- */

/* Start an algorithm: set every partition's vertex values to its initial
 * state — SSSP: d[source] = 0, else 0xFFFFFFFF; CC and LP: l[v] = v;
 * PageRank: r[v] = 1/N; personalized PageRank: r = e_source — and reset the
 * superstep counters. `source` is ignored for CC, LP and PageRank. LP builds
 * its row lists (in-degree classes; hub rows get hash tables of 2^k >= 2 x
 * in-degree slots) on first use. damping is used by
 * PageRank/PPR (e.g. 0.85). PPR runs the PageRank template (CONTRIB, SUM,
 * PAGERANK) with gxp_superstep(GXP_ALGO_PPR, ...). Builds the
 * partition caches (cached copies of remote sources, boundary set) on first
 * use. */
GXP_API gxp_status gxp_begin(gxp_ctx* ctx, gxp_algo algo, uint32_t source, float damping);

/* Copy the current values of the vertices owned by `part` (in local order,
 * n = owned count) to `out`: uint32 for SSSP/CC/LP, fp32 ranks for PageRank.
 * part = UINT32_MAX copies all partitions in global id order (n = n_vertices). */
GXP_API gxp_status gxp_get_values(gxp_ctx* ctx, uint32_t part, void* out, uint64_t n);

/* Overwrite the current values (same layout as gxp_get_values) and mark every
 * vertex changed, e.g. to resume from a checkpoint. Requires gxp_begin. */
GXP_API gxp_status gxp_set_values(gxp_ctx* ctx, uint32_t part, const void* in, uint64_t n);

/* ------------------------------------------------------------ superstep -- */

/* One superstep over every partition (Section IV-A1, BSP order Gen -> Merge
 * -> Apply): for each in-edge (u, v) of each owned vertex v, generate a
 * message from u's value (msggen), combine the messages by destination
 * (merge), then apply the result to v's value (apply), marking v in the
 * changed-vertex bitmap when its value changes. With more than one
 * partition it then synchronizes: each partition uploads only its changed
 * boundary vertices (lazy uploading, Algorithm 3) into the caches of the
 * others, and the exchange is skipped when there are none anywhere
 * (Section III-B3). Supported templates: SSSP = (RELAX, MIN, MIN),
 * CC = (LABEL, MIN, MIN), PageRank = (CONTRIB, SUM, PAGERANK),
 * LP = (LABEL, MODE, SET); others return
 * GXP_E_UNSUPPORTED. `algo` must match gxp_begin. If n_changed is non-NULL
 * the call waits for the device and stores the number of vertices whose
 * value changed; otherwise it returns once the work is enqueued. */
GXP_API gxp_status gxp_superstep(gxp_ctx* ctx, gxp_algo algo, gxp_msggen msggen,
                                 gxp_merge merge, gxp_apply apply, uint64_t* n_changed);

/* The global data queue entries of partition `part` from the last superstep
 * (Algorithm 3): the (id, value) pairs of its vertices that changed and are
 * cached by another partition, ascending by global id. *n_out receives the
 * count; if it exceeds `cap` nothing is copied and GXP_E_INVAL is returned.
 * *skipped (nullable) is 1 when the last exchange was skipped (no partition
 * had a changed boundary vertex). ids: uint32[cap]; vals: uint32 or fp32[cap].
 * Either of ids / vals may be NULL when cap is 0 (count query). */
GXP_API gxp_status gxp_sync(gxp_ctx* ctx, uint32_t part, uint32_t* ids, void* vals,
                            uint64_t cap, uint64_t* n_out, int* skipped);

/* The copies partition `part` holds in its cache now (Section III-B2,
 * LRU-based caching): their vertex ids, ascending, into ids[0 .. *n_out)
 * (host or device pointer). Without a budget (gxp_config.cache_slots = 0)
 * every remote source of the partition's in-edges is cached. With a budget
 * the cache starts empty at gxp_begin and, at every superstep boundary, the
 * copies the coming superstep uses (its frontier: vertices changed in the
 * superstep before; every vertex, or the source, before the first) enter it,
 * each copy's weight W <- min(65535, floor(W / 2) * cached + reads * used)
 * (reads: the partition's in-edges from that vertex), and the lowest weights
 * are evicted down to cache_slots, ties evicting the higher id. A used copy
 * that was not cached counts in gxp_stats.cache_downloads.
 * Errors: GXP_E_STATE (no graph loaded), GXP_E_INVAL (part out of range,
 * n_out NULL, or cap below the count, which *n_out then holds). */
GXP_API gxp_status gxp_cache_get(gxp_ctx* ctx, uint32_t part, uint32_t* ids, uint64_t cap, uint64_t* n_out);

/* Iteration control (Section II-C2): run supersteps until one changes no
 * vertex (SSSP, CC, LP) or max_steps of them (always max_steps for
 * PageRank; LP need not settle: the paper caps it at 15). Starts with
 * gxp_begin(algo, source, damping). *steps_done (nullable) counts supersteps
 * run, including the final one that changed nothing. SSSP and CC on one
 * partition run the loop on the device (a CUDA graph whose conditional
 * node repeats superstep + stop test, up to 32 supersteps per launch, one
 * host synchronization per launch); the others enqueue supersteps in
 * chunks and read their changed counts once per chunk. */
GXP_API gxp_status gxp_run(gxp_ctx* ctx, gxp_algo algo, uint32_t source, float damping,
                           uint32_t max_steps, uint32_t* steps_done);

GXP_API gxp_status gxp_stats_get(gxp_ctx* ctx, gxp_stats* out);

/* ------------------------------------------- batched multi-source SSSP -- */

typedef struct gxp_batch_opts {
    uint32_t streamed;       /* 1: edges stay in pinned host memory and every superstep
                                streams them through a ring of device buffers (the pipeline
                                shuffle of Section III-A, Algorithms 1-2); 0: edges resident */
    uint32_t pipelined;      /* streamed only: 1 = copy of block i+1 overlaps compute of block
                                i (3-slot ring); 0 = copy, then compute, block by block */
    uint64_t block_edges;    /* streamed only: edges per block; 0 = choose by the Lemma 1 model
                                from measured coefficients, then a local sweep (autotuner) */
    uint32_t use_graph;      /* 1: replay each superstep from a captured CUDA graph */
    uint32_t max_steps;      /* 0 = run to convergence */
    const char* tune_cache;  /* path of the autotuner's JSON cache, or NULL: with block_edges = 0
                                a record for this graph shape and GPU (gxp_tune_cache_get) is
                                used instead of measuring, and a new measurement is stored */
    uint32_t reserved[4];
} gxp_batch_opts;

typedef struct gxp_batch_report {
    uint32_t supersteps;     /* supersteps run, including the final one that changed nothing */
    uint32_t blocks;         /* edge blocks per superstep (streamed) */
    uint64_t block_edges;    /* edges per block used */
    double   ms_total;       /* wall time of the run on the device stream, excluding set-up */
    double   k1, k2, k3, a;  /* autotuner: per-edge download/compute/upload and per-block cost (ms) */
    double   model_block_edges;  /* Lemma 1's continuous optimum b_opt (edges) */
    double   model_ms;       /* the pipeline-time equation's estimate at the chosen block size */
    double   sweep_best_ms;  /* measured superstep time at the chosen block size (autotuner) */
    uint64_t edges_per_superstep;
    uint64_t tune_from_cache;   /* 1: the coefficients and block size came from the tune cache */
    uint64_t active_edges;      /* in-edges whose source was in the frontier, summed over the
                                   supersteps (each gathered a 256-byte distance row) */
    uint64_t persistent;        /* 1: resident edges, the whole run in one persistent
                                   cooperative kernel (grid barrier between supersteps) */
    uint64_t reserved[3];
} gxp_batch_report;

/* One autotuner record (Section III-A): the per-edge download, compute and
 * upload costs k1, k2, k3 and the per-block cost a (ms), Lemma 1's continuous
 * optimum, the block size the local sweep chose and its measured superstep
 * time. */
typedef struct gxp_tune_record {
    double k1, k2, k3, a;
    double model_block_edges;
    double block_edges;
    double sweep_best_ms;
} gxp_tune_record;

/* The autotuner's cache file (JSON: one member per key). The key the batch
 * engine uses is "sssp_batch V=<vertices> E=<edges> deg=<floor(log2(E/V))>
 * esize=<bytes per streamed edge> gpu=<device name>". get: GXP_OK and *out
 * when the file holds the key, GXP_E_INVAL when it does not (or the file is
 * missing); put: adds or replaces the member (the file is rewritten through a
 * temporary and renamed), GXP_E_INVAL if it cannot be written. Host-only:
 * neither touches the GPU. */
GXP_API gxp_status gxp_tune_cache_get(const char* path, const char* key, gxp_tune_record* out);
GXP_API gxp_status gxp_tune_cache_put(const char* path, const char* key, const gxp_tune_record* rec);

/* Multi-source Bellman-Ford (Section V-A runs several SSSP sources at once):
 * n_sources <= 64 sources advance together, every edge serving all of them.
 * Requires a single-partition weighted graph. dist_out (host or device,
 * nullable) receives uint32[n_vertices][n_sources]: dist_out[v*n_sources+s]
 * is the distance from sources[s] to v (0xFFFFFFFF if unreachable) — equal,
 * source by source, to gxp_run(GXP_ALGO_SSSP). opts may be NULL (resident
 * edges, run to convergence); report may be NULL. */
GXP_API gxp_status gxp_sssp_batch(gxp_ctx* ctx, const uint32_t* sources, uint32_t n_sources,
                                  uint32_t* dist_out, const gxp_batch_opts* opts,
                                  gxp_batch_report* report);

/* -------------------------------------------------------------- serving -- */

/* Continuous batching of queries over graphs resident on the device (the
 * paper has no serving layer; this follows its multi-query use of one pass
 * over the edges, Section V-A). Each served graph has one lane per query
 * kind; a lane runs up to 64 queries as the columns of one [V][64] state
 * matrix, so every superstep's pass over the edges serves all of them.
 * Queries that arrive while others run are admitted at the next superstep
 * boundary once a slot and a result buffer are free (admission by memory: a
 * query holds one device result buffer of n_vertices x 4 bytes from
 * admission until its result is collected). A query's result does not
 * depend on which other queries share its supersteps: every slot computes
 * from its own column in an order fixed by the edge order, so results are
 * bit-identical alone and in any mix.
 *
 * Threading: gxp_query_submit, gxp_query_poll, gxp_query_next_done,
 * gxp_query_info_get and gxp_serve_report_get may be called from any number
 * of threads at once; gxp_serve_add_graph, gxp_serve_start and
 * gxp_serve_stop from one thread while no other call on the server runs.
 * These calls report error details through gxp_last_error(NULL) on the
 * calling thread; they do not touch the context's superstep engine. */

typedef enum gxp_query_kind {
    GXP_QUERY_SSSP = 0,     /* Bellman-Ford distances from `source` (weighted graphs) */
    GXP_QUERY_PPR = 1       /* personalized PageRank from `source`: r_0 = e_s,
                               r_{t+1} = d A^T D^-1 r_t + ((1-d) + d D_t) e_s, where D_t is the
                               mass of r_t on vertices without out-edges; fp32 ranks, exact
                               fixed-point D_t; `iters` supersteps */
} gxp_query_kind;

typedef enum gxp_query_state {
    GXP_QUERY_QUEUED = 0, GXP_QUERY_RUNNING = 1, GXP_QUERY_DONE = 2, GXP_QUERY_FAILED = 3
} gxp_query_state;

typedef struct gxp_serve_opts {
    uint32_t max_slots;          /* queries run at once per (graph, kind), 1..64; 0 = 64 */
    uint32_t results_per_graph;  /* device result buffers per graph; 0 = 2 * max_slots */
    uint32_t queue_cap;          /* queries waiting for admission, all graphs; 0 = 2^20 */
    uint32_t priorities;         /* 1: lanes of graphs with fewer edges get higher CUDA stream
                                    priority (their short supersteps overtake long ones at block
                                    boundaries); 0: equal priority */
    uint32_t reserved[8];
} gxp_serve_opts;

typedef struct gxp_query_info {
    uint32_t state;              /* gxp_query_state */
    uint32_t supersteps;         /* supersteps the query took part in */
    uint32_t graph;
    uint32_t kind;               /* gxp_query_kind */
    uint64_t n_values;           /* result length: n_vertices of the graph */
    double   queue_ms;           /* submission -> admission */
    double   run_ms;             /* admission -> result ready on the device */
    uint64_t reserved[4];
} gxp_query_info;

typedef struct gxp_serve_report {
    uint64_t submitted, completed, failed;
    uint64_t queued, running;    /* now */
    uint64_t sssp_supersteps;    /* over all graphs since gxp_serve_start */
    uint64_t ppr_supersteps;
    uint64_t device_bytes;       /* held by the server */
    uint64_t reserved[8];
} gxp_serve_report;

/* Make a graph resident for serving: n_edges directed edges src[i] -> dst[i]
 * (uint32 ids < n_vertices), weights uint32 (NULL: the graph serves PPR
 * only). Arrays may be host or device pointers and are copied. *graph
 * receives the graph's index (0, 1, ... in order of addition). Only before
 * gxp_serve_start. Errors: GXP_E_INVAL (ids, sizes, more than 2^32 - 1
 * edges), GXP_E_NOMEM (over the context's mem_budget, which bounds the
 * server's device memory), GXP_E_STATE (server running). */
GXP_API gxp_status gxp_serve_add_graph(gxp_ctx* ctx, uint64_t n_vertices, uint64_t n_edges,
                                       const uint32_t* src, const uint32_t* dst,
                                       const uint32_t* weights, uint32_t* graph);

/* Allocate the lanes and result pools and start one host thread per lane.
 * opts may be NULL. Errors: GXP_E_NOMEM, GXP_E_STATE (no graph / running). */
GXP_API gxp_status gxp_serve_start(gxp_ctx* ctx, const gxp_serve_opts* opts);

/* Stop the lanes: queued and running queries fail with GXP_E_STATE; results
 * already done stay collectable. The server can be started again. */
GXP_API gxp_status gxp_serve_stop(gxp_ctx* ctx);

/* Queue a query. damping in [0, 1) (PPR only), iters = PPR supersteps
 * (0 = 20); both are ignored for SSSP, which runs until no distance of the
 * query improves. *qid receives its id (never 0). Errors: GXP_E_INVAL
 * (graph, kind, source, damping), GXP_E_UNSUPPORTED (SSSP on an unweighted
 * graph), GXP_E_BUSY (queue_cap queries already waiting), GXP_E_STATE (not
 * started, or a lane failed). */
GXP_API gxp_status gxp_query_submit(gxp_ctx* ctx, uint32_t graph, gxp_query_kind kind,
                                    uint32_t source, float damping, uint32_t iters, uint64_t* qid);

/* Wait up to timeout_ms (0: do not wait, < 0: without limit) for query qid.
 * *done = 1 once its result is ready. Then, if out is non-NULL, the result
 * (uint32 distances, 0xFFFFFFFF = unreachable, or fp32 ranks; n_vertices
 * values, cap must be at least that) is copied to out (host or device
 * memory) and the query is released: its id becomes invalid and its result
 * buffer returns to the pool. With out = NULL the query stays. A failed
 * query returns its error (and is released when out is non-NULL).
 * Errors: GXP_E_INVAL (unknown qid, cap too small). */
GXP_API gxp_status gxp_query_poll(gxp_ctx* ctx, uint64_t qid, void* out, uint64_t cap,
                                  int timeout_ms, int* done);

/* Wait up to timeout_ms (< 0: without limit) for a finished (done or failed)
 * query not yet handed out by this call, in order of completion. *qid
 * receives its id, or 0 on timeout. */
GXP_API gxp_status gxp_query_next_done(gxp_ctx* ctx, int timeout_ms, uint64_t* qid);

/* State and timing of a query not yet released. */
GXP_API gxp_status gxp_query_info_get(gxp_ctx* ctx, uint64_t qid, gxp_query_info* out);

GXP_API gxp_status gxp_serve_report_get(gxp_ctx* ctx, gxp_serve_report* out);

/* ----------------------------------------------- block-size model (a8) -- */

/* Lemma 1 (Section III-A, "Block Size Selection"): with per-entity download,
 * compute and upload costs k1, k2, k3, per-block call cost a and d entities,
 * return the integer block size *b and count *s (s >= 2) that minimise the
 * pipeline-time equation among the rounded candidates floor/ceil(s_opt) and
 * floor/ceil(b_opt), and the equation's estimate *t. Host-only arithmetic. */
GXP_API gxp_status gxp_block_size_model(double k1, double k2, double k3, double a, uint64_t d,
                                        uint64_t* b, uint64_t* s, double* t);

/* ------------------------------------------ allocation-free superstep -- */

/* The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory themselves — for example
 * code whose GPU memory is wholly owned by another allocator (a framework's
 * caching pool), or latency-sensitive code that cannot accept cudaMalloc's
 * implicit device synchronisation.
 *
 * One SSSP (RELAX, MIN, MIN) or CC (LABEL, MIN, MIN) superstep over a single
 * partition's CSC that lives in the caller's device memory, computing d_next
 * from d_cur exactly as gxp_superstep does. It calls no cudaMalloc, cudaFree
 * or allocating library routine. Its scratch is a fixed file-scope device
 * array of about 6.8 MB that every GPU loading libgxp.so holds until the
 * process exits; it limits the input to 4 * n_vertices + n_edges <= 2^28
 * (larger inputs return GXP_E_INVAL).
 *
 * Arguments (all device pointers, on the current CUDA device):
 *   d_col_ptr  uint32[n_vertices + 1], CSC offsets from 0 to n_edges
 *   d_src      uint32[n_edges] source ids (< n_vertices), dst-sorted
 *   d_w        uint32[n_edges] weights (SSSP only; NULL for CC)
 *   d_cur      uint32[n_vertices] current values (read only)
 *   d_next     uint32[n_vertices] next values (written); must not overlap
 *              d_cur (GXP_E_INVAL)
 * d_col_ptr, d_src, d_w and d_cur must be 16-byte aligned and readable up to
 * round_up(n_vertices + 1, 4), round_up(n_edges, 4) and round_up(n_vertices, 4)
 * elements. n_changed
 * (host pointer, nullable) receives the number of vertices whose value
 * changed. The call is enqueued on `stream` (a cudaStream_t, NULL = default
 * stream) and waits for it before returning.
 *
 * The first call on a device looks up the scratch's device address (once per
 * device); make that first call before any stream capture. Every call clears
 * the parts of the scratch that must start at zero, but all calls share the
 * one array: calls that overlap on the GPU race and give wrong results.
 * Before any edge block is cut, a kernel checks the CSC on the device (the
 * call waits for it): offsets that do not run from 0 to n_edges without
 * decreasing return GXP_E_INVAL, a source id >= n_vertices GXP_E_BOUNDS, and
 * nothing else runs. The kernel's bounded waits on its bulk copies return
 * GXP_E_TIMEOUT when they run out (GXP_FAULT=timeout makes every wait give
 * up at once, to test that path); a warp that gives up first waits for its
 * own copies in flight.
 * Errors: GXP_E_INVAL (sizes, null, misaligned or overlapping pointers,
 * input beyond the scratch limit, CSC offsets out of order),
 * GXP_E_UNSUPPORTED (other algorithms), GXP_E_BOUNDS (a source id out of
 * range), GXP_E_TIMEOUT, GXP_E_CUDA. */
GXP_API gxp_status gxp_superstep_min_noalloc(gxp_algo algo, uint32_t n_vertices, uint64_t n_edges,
                                             const uint32_t* d_col_ptr, const uint32_t* d_src,
                                             const uint32_t* d_w, const uint32_t* d_cur,
                                             uint32_t* d_next, uint64_t* n_changed, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GXP_H */
