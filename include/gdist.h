/*
 * gdist.h -- C ABI of the GB300 mesh-mesh distance engine.
 *
 * The engine computes, for two triangle meshes placed by rigid transforms,
 *   D_min = min ||p - q||  and  D_max = max ||p - q||  over p in mesh A, q in
 *   mesh B (the paper's problem statement: Section 3, Eqs. 1-2),
 * with a bounding-volume-pair (BVTT) front traversal over full binary
 * "f12" BVHs (Section 7.3), pruned against a shared running bound computed
 * from the AABB distance bounds of Section 4 (Eqs. 5-11), followed by an
 * exact triangle-triangle narrow phase on the surviving pairs.  Traversal and
 * culling run in float32 with outward-widened bounds; the final candidates are
 * re-evaluated in float64.
 *
 * Conventions shared by every entry point:
 *   - Vertices are float32 xyz triples; triangles are int32 index triples.
 *   - Transforms are 12 doubles, a row-major 3x4 matrix [R | t] that maps
 *     local coordinates v to world coordinates R v + t.  R must be orthonormal
 *     to within 1e-9 (max-abs entry of R^T R - I); otherwise GD_ERR_INVALID_ARG.
 *   - Results are in world units.  Witness triangles are the caller's original
 *     triangle indices; witness points are float64 world coordinates.
 *   - Every host pointer argument is read (or written) during the call only;
 *     the library copies what it keeps.  Handles are owned by the library and
 *     released by the matching *_destroy / gd_serve_stop call.  A mesh must
 *     outlive every query and server that uses it, and the context must outlive
 *     its meshes.
 *   - Thread safety: a gd_ctx serves one host thread at a time (serialise
 *     calls on a shared context); a gd_server may be used from any thread.
 *   - No entry point falls back to a CPU computation: without a CUDA device
 *     gd_ctx_create fails with GD_ERR_CUDA.
 */
#ifndef GDIST_H_
#define GDIST_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GD_API __attribute__((visibility("default")))
#else
#define GD_API
#endif

typedef enum {
    GD_OK = 0,
    GD_ERR_INVALID_ARG = 1, /* a NULL handle, bad sizes, out-of-range indices,
                               non-finite data, or a non-orthonormal R */
    GD_ERR_OOM = 2,         /* device or pinned host allocation failed */
    GD_ERR_CUDA = 3,        /* a CUDA runtime error (text in gd_last_error) */
    GD_ERR_NOT_BUILT = 4,   /* query on a mesh whose BVH was not built */
    GD_ERR_OVERFLOW = 5,    /* a work queue exceeded its capacity even after
                               the library grew it to the configured limit */
    GD_ERR_TIMEOUT = 6,     /* a bounded device wait gave up (the kernel
                               returned early; the context stays usable) */
    GD_ERR_BUSY = 7,        /* server: request not admitted (no slot / memory) */
    GD_ERR_NOT_READY = 8    /* server: ticket not finished yet */
} gd_status;

typedef enum { GD_MIN = 0, GD_MAX = 1 } gd_kind;

typedef struct gd_ctx gd_ctx;
typedef struct gd_mesh gd_mesh;
typedef struct gd_server gd_server;

/* One query answer.  For GD_MIN, pa and pb are a closest pair (pa on tri_a
 * of mesh A, pb on tri_b of mesh B); for GD_MAX, a farthest vertex pair.
 * status is a gd_status for this query; flags bit 0 = meshes intersect
 * (d == 0); flags bit 1 = the traversal stopped early because a triangle pair
 * at float64 distance exactly 0 was found (Section 8: with penetration the
 * minimum distance is zero).  The witness of d > 0 is the pair at the extreme
 * with the smallest (tri_a, tri_b); the witness of d == 0 is that first
 * proving pair, any intersecting pair, and may differ between runs. */
typedef struct {
    double d;
    int64_t tri_a, tri_b;
    double pa[3], pb[3];
    uint32_t status, flags;
} gd_result;

/* Answer of the naive comparator (gd_naive_query). */
typedef struct {
    double d;                  /* float32 distance (squared in float32, root taken in float64) */
    uint64_t node_tests;       /* (triangle of A, node of B) box tests: the BVTT nodes visited */
    uint64_t leaf_tests;       /* triangle pairs evaluated */
    uint64_t max_thread_tests; /* most box tests of one thread (load imbalance) */
    uint32_t status;           /* GD_OK, or GD_ERR_TIMEOUT (d and the counts are partial) */
    uint32_t pad;
} gd_naive_result;

/* Answer of a point-to-mesh query (gd_point_distance). */
typedef struct {
    double d;        /* float64 distance from the point to the mesh surface */
    int64_t tri;     /* the caller's index of the closest triangle (smallest among ties) */
    double p[3];     /* closest point on that triangle, world frame */
    uint32_t status; /* GD_OK; GD_ERR_INVALID_ARG (non-finite point); GD_ERR_TIMEOUT */
    uint32_t pad;
} gd_point_result;

/* One query of a batch or of the server. */
typedef struct {
    const gd_mesh *a, *b;
    double xa[12], xb[12];
    gd_kind kind;
    uint64_t user_tag;
} gd_query;

/* BVH build options (NULL = defaults). */
typedef struct {
    int morton_bits; /* bits per axis of the Morton code, 1..21 (default 21) */
} gd_build_opts;

/* Traversal tunables of a context.  Zero fields keep the current value. */
typedef struct {
    int64_t work_target;   /* C of Section 6: a level expands n front entries by
                              k levels per side with n * 4^k < C (default 2^17) */
    int32_t k_max;         /* cap on k (default 6) */
    int32_t blocks_per_sm; /* persistent CTAs per SM (default: occupancy limit) */
    int64_t front_capacity;/* BVTT entries per front buffer (default 2^24) */
    int64_t leaf_capacity; /* leaf-pair queue entries (default 2^24) */
    int64_t cand_capacity; /* float64 candidate slots (default 2^22) */
    int64_t max_capacity;  /* growth limit for the three above (default 2^30) */
    int64_t timeout_ns;    /* bound on every device-side wait (default 2e9) */
    int32_t refit_mode;    /* 1: refit B's low subtrees (2^8 leaves) into A's
                              frame when the front first reaches them (default);
                              2: never, bound B's local boxes under the map;
                              3: refit all of B into A's frame at the start of
                              every single query, the paper's per-frame refit
                              of Section 8 (batches, the server and
                              gd_query_device_noalloc, which has no room for a
                              whole tree, then run as 2).  Same results in
                              every mode */
    int32_t refit_slots;   /* subtrees refit per launch (default 2^13) */
    int32_t probes;        /* greedy probes that seed the running bound
                              (default 64).  Single queries: they start at the
                              root in up to grid/8 extra CTAs (8 probes each)
                              that run beside the traversal; batches: after
                              the first refit, at least one per query.  A min
                              query's repeated probes on fronts beyond 4 C use
                              at least 256 */
    int64_t batch_budget;  /* batches: room per query and level in the first
                              round (default 2^23); a launch takes max_capacity
                              / (2 x budget) queries; half of the room is each
                              query's own share, the other half a pool common
                              to the launch; a query that pushes more than its
                              share in one level draws on the pool, and when
                              the pool is spent leaves the launch for the next
                              round, whose budget is 16x larger (chunks 16x
                              smaller); a chunk of one runs alone */
    int32_t bounds_mode;   /* 1: enhanced bounds, Eq. 10 (upper bound of the
                              min) and Eq. 11 (lower bound of the max), the
                              default; 2: conventional bounds only, Eq. 9 (the
                              farthest-point bound) for the min and the box gap
                              for the max: the ablation of Section 9, same
                              results, more node pairs */
} gd_tunables;

/* Counters of the last query (or batch) run on a context. */
typedef struct {
    uint32_t levels;             /* BVTT expansion levels executed */
    uint32_t front[32];          /* front entries entering each level */
    uint32_t slots[32];          /* log2 descendant pairs per entry per level */
    uint64_t pairs_tested;       /* BVH node pairs whose bounds were computed */
    uint32_t leaf_pairs;         /* leaf-leaf pairs reaching the narrow phase */
    uint32_t tri_pairs;          /* float32 triangle pairs evaluated */
    uint32_t candidates;         /* triangle pairs kept for float64 refinement */
    uint32_t refined;            /* candidates evaluated in float64 */
    uint64_t alg_bytes;          /* algorithmic bytes moved by the traversal
                                    kernel (front entries, node boxes, triangles,
                                    candidates), counted by the kernel */
    uint32_t retries;            /* capacity growths during the call */
    uint32_t blocks;             /* persistent CTAs launched */
    uint32_t level_ns[32];       /* device time of each expansion level */
    uint32_t phase_ns[12];       /* device time of: setup, subtree refits, probes,
                                    all levels, leaf narrow phase, float64
                                    refinement, wait for the refinement of the
                                    other CTAs, witness selection, result
                                    records, total, (2 unused); CTA 0's view;
                                    after gd_batch_query, summed over its
                                    launches */
    uint32_t probes;             /* greedy descents run to seed the bound */
    float u_level[32];           /* running bound entering each level (query 0) */
    float u_probe;               /* running bound after the probes (query 0) */
    uint32_t refits;             /* B subtrees refit into A's frame */
} gd_stats;

/* ---- context ----------------------------------------------------------- */

/* Create a context on CUDA device `device`; allocates its stream and, on the
 * first query, its work buffers.  GD_ERR_CUDA if the device is unusable. */
GD_API gd_status gd_ctx_create(int device, gd_ctx **out);
GD_API void gd_ctx_destroy(gd_ctx *ctx);
/* Message of the last failing call on ctx ("" if none).  Owned by ctx. */
GD_API const char *gd_last_error(gd_ctx *ctx);
GD_API gd_status gd_ctx_set_tunables(gd_ctx *ctx, const gd_tunables *t);
/* Autotuner (no counterpart in the paper): times the caller's sample (one
 * query, or a batch of n, run as gd_min/max_distance or gd_batch_query) under
 * settings of work_target, k_max, probes, blocks_per_sm and, for n > 1,
 * batch_budget, one coordinate-descent pass (median of reps timed runs after
 * one untimed run per setting; a value is kept when >= 1% faster), and leaves
 * the fastest setting in ctx (also copied to *best unless NULL).  Tunables
 * change the speed only, never a result.  Synchronous; errors of the sample's
 * queries are returned (the tunables then stay as they were before the
 * failing setting). */
GD_API gd_status gd_autotune(gd_ctx *ctx, const gd_query *sample, int64_t n, int32_t reps, gd_tunables *best);
GD_API gd_status gd_ctx_get_tunables(gd_ctx *ctx, gd_tunables *t);
GD_API gd_status gd_get_stats(gd_ctx *ctx, gd_stats *out);
/* The CUDA stream (cudaStream_t) the context runs on. */
GD_API void *gd_ctx_stream(gd_ctx *ctx);

/* ---- meshes (Section 7.3: f12-BVH) --------------------------------------- */

/* Copy a mesh to the device.  verts: nv x 3 float32 (host), tris: nt x 3 int32
 * (host), 1 <= nt <= 2^30.  Indices must lie in [0, nv) and every vertex must
 * be finite (checked on the device by gd_bvh_build). */
GD_API gd_status gd_mesh_create(gd_ctx *ctx, const float *verts, int64_t nv, const int32_t *tris,
                                int64_t nt, gd_mesh **out);
/* Build the mesh's f12-BVH on the device (Section 7.3): Morton codes of the
 * triangle centroids, a stable radix sort (ties by original index), 2^L
 * leaves (L = floor(log2 nt)) of one or two consecutive sorted triangles, leaf
 * boxes that are exact bounds of their vertices, and a level-by-level union of
 * boxes up to the root.  Every box is tight (Section 4, tightness lemma).
 * Synchronous.  GD_ERR_INVALID_ARG on bad indices or non-finite vertices. */
GD_API gd_status gd_bvh_build(gd_mesh *mesh, const gd_build_opts *opts);
/* Deformable meshes (Section 8: the BVH is refit on the fly when vertices
 * move).  Replaces the vertex positions of a built mesh (same count nv, same
 * triangles) and refits its tree on the device: the leaf order of the last
 * gd_bvh_build is kept, leaf boxes are recomputed as exact bounds of the new
 * vertices and every inner box as the union of its children, so every box is
 * tight again and queries stay exact.  Only the culling efficiency depends on
 * how far the mesh moved since the build (call gd_bvh_build to re-sort).
 * verts: nv x 3 float32, host or device memory (read before the call
 * returns).  Synchronous on the context's stream; queries on the context's
 * stream see the new positions.  The caller must not update a mesh while a
 * query that uses it is in flight on another stream (a server's, a captured
 * graph's).  GD_ERR_NOT_BUILT if the mesh has no tree; GD_ERR_INVALID_ARG if
 * nv differs from the mesh's or a coordinate is not finite (the mesh is then
 * left unbuilt until the next successful update or build). */
GD_API gd_status gd_mesh_update(gd_mesh *mesh, const float *verts, int64_t nv);
GD_API void gd_mesh_destroy(gd_mesh *mesh);
/* Device time in ms of the kernels of the mesh's last gd_bvh_build (index
 * validation, Morton codes, radix sort, leaves and level reduction; CUDA
 * events on the context's stream around them, allocations excluded).
 * Preprocessing: the paper times its builds apart from the queries (Section
 * 8).  GD_ERR_NOT_BUILT for a mesh without a tree. */
GD_API gd_status gd_mesh_build_time(const gd_mesh *mesh, double *device_ms);
/* Tree depth L (leaves = 2^L) and triangle count of a built mesh. */
GD_API gd_status gd_mesh_info(const gd_mesh *mesh, int32_t *levels, int64_t *triangles);
/* Copy the BVH to the host for inspection: boxes (6 floats per node, node
 * ids 1 .. 2^(L+1)-1 in heap order, entry 0 unused) and the original index of
 * each triangle in leaf order.  Either pointer may be NULL. */
GD_API gd_status gd_mesh_download(const gd_mesh *mesh, float *boxes, int32_t *tri_order);

/* ---- queries (Algorithms 1-2; Sections 5-7) ------------------------------ */

/* Minimum distance D_min (Eq. 1).  xa, xb: host transforms.  Synchronous:
 * the transforms travel as launch parameters, one persistent traversal
 * launch runs, and its last CTA writes the result record to the context's
 * pinned host memory, which the call waits for (bounded by the launch's own
 * completion; no stream synchronisation on the way back). */
GD_API gd_status gd_min_distance(gd_ctx *ctx, const gd_mesh *A, const gd_mesh *B, const double xa[12],
                                 const double xb[12], gd_result *out);
/* Maximum distance D_max (Eq. 2); same contract as gd_min_distance. */
GD_API gd_status gd_max_distance(gd_ctx *ctx, const gd_mesh *A, const gd_mesh *B, const double xa[12],
                                 const double xb[12], gd_result *out);
/* Point-to-mesh distances (Eq. 1 with one side a single point; the 1-to-N
 * direction of Section 10's future work, with N query points): for each of
 * n world points, the closest point of mesh M placed by x (12 doubles, as
 * for the mesh queries).  Exact in float64: one thread per point walks M's
 * tree once in float32 with a running bound that is always a true upper
 * bound (each triangle's float32 closest point, widened for the float32
 * errors), and takes the float64 distance of every triangle whose rigorous
 * float32 lower bound is within it, so the result is the minimum over all
 * triangles, the smallest index among ties.  points: n x 3 float64; points
 * and out may each be host or device memory.  Synchronous.  Per-point
 * status in out; the call returns GD_ERR_TIMEOUT if some point passed the
 * context's timeout. */
GD_API gd_status gd_point_distance(gd_ctx *ctx, const gd_mesh *M, const double x[12], const double *points,
                                   int64_t n, gd_point_result *out);
/* Work of the context's last gd_point_distance call: node boxes tested and
 * float64 point-triangle distances taken, summed over its points. */
GD_API gd_status gd_point_stats(gd_ctx *ctx, uint64_t *node_tests, uint64_t *exact_tests);
/* The naive GPU comparator of Section 8 (Performance): one thread per
 * triangle of A walks B's BVH depth first (nearer child first), pruning with
 * the conventional box bounds (Eqs. 5-8) against one global running bound
 * read and updated with atomics; float32 throughout.  Not the product path:
 * it exists to measure the BVTT nodes such a walk visits and its load
 * imbalance against the front traversal.  Same meshes and transforms as
 * gd_min_distance; kind GD_MIN or GD_MAX.  timeout_ns > 0 bounds the launch
 * (0: the context's timeout): threads stop at the deadline and the call
 * returns GD_ERR_TIMEOUT with out filled in (partial counts, d an upper
 * (min) or lower (max) bound).  Synchronous. */
GD_API gd_status gd_naive_query(gd_ctx *ctx, const gd_mesh *A, const gd_mesh *B, gd_kind kind,
                                const double xa[12], const double xb[12], int64_t timeout_ns,
                                gd_naive_result *out);
/* Device-resident form: d_xa, d_xb are device pointers to 12 doubles each,
 * d_out a device pointer to one gd_result; stream is a cudaStream_t (NULL =
 * the context's stream).  Asynchronous (no host synchronisation); the
 * context's work buffers must already be sized (any prior synchronous query
 * does that).  Returns launch errors only; the per-query status is in
 * d_out->status. */
GD_API gd_status gd_query_device(gd_ctx *ctx, const gd_mesh *A, const gd_mesh *B, gd_kind kind,
                                 const double *d_xa, const double *d_xb, gd_result *d_out, void *stream);
/* Device-resident query that allocates nothing (the paper has no counterpart:
 * this is for callers that must not allocate device memory while they run,
 * such as a per-frame control loop where a cudaMalloc could stall or fail, or
 * a process whose device memory is held by another allocator).  Same inputs
 * and output as gd_query_device (device pointers; stream is a cudaStream_t,
 * NULL = the legacy default stream); A and B must belong to one context,
 * and the calling thread's current CUDA device must be that context's device
 * (otherwise GD_ERR_INVALID_ARG; the call never changes the current device).
 * The context's tunables (bounds, refit mode, probes, work target, k_max,
 * timeout) are applied exactly as gd_query_device applies them, so both give
 * the same traversal.  Every work buffer comes from one 32 MiB array compiled
 * into the library (held by every GPU that loads the library, until exit).
 * The first call on a device looks up that array's device address: make it
 * before any stream capture.  Limits: with refit on, B with at most 24 tree
 * levels (fewer than 2^25 triangles; larger B: GD_ERR_INVALID_ARG); at most
 * 2^18 front entries, 2^18 leaf pairs and 2^16 float64 candidates per call
 * (beyond them d_out->status is GD_ERR_OVERFLOW: use gd_query_device).
 * Errors: GD_ERR_INVALID_ARG (NULL pointer, bad kind, meshes of two
 * contexts, wrong current device, B too deep), GD_ERR_NOT_BUILT (a mesh
 * without a tree), GD_ERR_CUDA (launch failure).  Calls share the array:
 * calls whose work overlaps on the GPU race, so serialise them.
 * Asynchronous; returns argument and launch errors only. */
GD_API gd_status gd_query_device_noalloc(const gd_mesh *A, const gd_mesh *B, gd_kind kind, const double *d_xa,
                                         const double *d_xb, gd_result *d_out, void *stream);
/* A captured CUDA graph of one device-resident query (the launch of
 * gd_query_device with these arguments), for loops that ask the same
 * question every frame: update *d_xa / *d_xb in place (device memory), then
 * gd_graph_launch; the result lands in *d_out as for gd_query_device
 * (status GD_ERR_OVERFLOW when the work outgrew the buffers: run one
 * synchronous query to grow them).  The graph holds one cooperative kernel
 * node; it is rebuilt by gd_graph_launch when the context's work buffers or
 * tunables changed.  Meshes, transforms and result must outlive the graph.
 * No counterpart in the paper. */
typedef struct gd_graph gd_graph;
GD_API gd_status gd_graph_create(gd_ctx *ctx, const gd_mesh *A, const gd_mesh *B, gd_kind kind, const double *d_xa,
                                 const double *d_xb, gd_result *d_out, gd_graph **out);
/* Asynchronous on stream (NULL: the context's stream). */
GD_API gd_status gd_graph_launch(gd_graph *g, void *stream);
GD_API gd_status gd_graph_destroy(gd_graph *g);

/* n independent queries (any mix of meshes and kinds), results in
 * out[0..n).  Synchronous.  Each kind runs in persistent launches of chunks
 * of queries whose fronts share the work queues (sizes: see batch_budget in
 * gd_tunables); a query whose fronts outgrow its share leaves its launch and
 * runs again in a later, smaller chunk, finally alone with grown buffers.
 * Results equal those of single queries (the d = 0 witness may differ, see
 * gd_result). */
GD_API gd_status gd_batch_query(gd_ctx *ctx, const gd_query *q, int64_t n, gd_result *out);

/* Completion times of the queries of the last gd_batch_query on ctx (no
 * counterpart in the paper): done_ns[i] = device-clock nanoseconds from the
 * start of that call's first launch to the moment the kernel wrote query i's
 * final result record (for a query rerun in a later launch, that launch's
 * record).  Stamps come from the GPU's global timer, so host overheads
 * before the first launch are not counted.  n must equal the batch's query
 * count (else GD_ERR_INVALID_ARG); done_ns: n int64 values (host). */
GD_API gd_status gd_batch_times(gd_ctx *ctx, int64_t n, int64_t *done_ns);

/* ---- serving ----------------------------------------------------------- */

typedef struct {
    int32_t slots;            /* ignored (kept for layout): the server runs one
                                 launch at a time on the whole GPU, since CUDA
                                 does not promise that cooperative grids
                                 launched on different streams are resident
                                 together */
    int32_t max_batch;        /* queries per launch (default 16) */
    int64_t memory_budget;    /* bytes of work buffers of the server's lane
                                 (default 8 GiB); requests are admitted while
                                 the predicted footprints of the queued and
                                 running ones stay within it */
    int32_t linger_us;        /* wait this long for more requests before
                                 launching a partial batch (default 0) */
} gd_serve_opts;

/* Predicted work-buffer bytes of one query (the server's admission model:
 * power laws in sqrt(T_A) + sqrt(T_B) fitted as upper envelopes of the front,
 * leaf-pair and candidate peaks measured on single queries).  No counterpart
 * in the paper; its memory analysis (Section 8) separates the static BVH
 * memory from the dynamic front memory that this predicts. */
GD_API gd_status gd_query_footprint(const gd_query *q, int64_t *bytes);

/* Start a server on ctx's device (continuous batching: a serving thread takes
 * all queued requests of the oldest request's kind, up to max_batch and
 * within the memory budget, into one persistent launch on the whole GPU, and
 * requests that arrive meanwhile join the next launch as soon as it ends; a
 * lone request runs as a single query).  The server has its own stream and
 * work buffers (sized from memory_budget, allocated here); ctx is used only to
 * validate submissions and must outlive the server. */
GD_API gd_status gd_serve_start(gd_ctx *ctx, const gd_serve_opts *opts, gd_server **out);
/* Enqueue one query; GD_ERR_BUSY if the queue is full (max(4096, 16 x
 * max_batch) waiting requests) or if its predicted footprint
 * (gd_query_footprint) would take the footprints held by queued and running
 * requests beyond the memory budget (a request's footprint is held from
 * submission until its result is ready; a request larger than the whole
 * budget is admitted only when nothing else is held, and runs alone with
 * buffers grown for it).  *ticket identifies the request. */
GD_API gd_status gd_serve_submit(gd_server *srv, const gd_query *q, uint64_t *ticket);
/* GD_OK and *out filled if the ticket is done (the ticket is then released);
 * GD_ERR_NOT_READY otherwise. */
GD_API gd_status gd_serve_poll(gd_server *srv, uint64_t ticket, gd_result *out);
/* Up to max finished requests (any tickets): their tickets in tickets[0..*n)
 * and results in out[0..*n); those tickets are released.  GD_OK with *n = 0
 * when none is finished. */
GD_API gd_status gd_serve_drain(gd_server *srv, uint64_t *tickets, gd_result *out, int64_t max, int64_t *n);
/* Drain in-flight work, stop the loop and free the server. */
GD_API gd_status gd_serve_stop(gd_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* GDIST_H_ */
