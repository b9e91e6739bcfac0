/*
 * gwn.h - C ABI of the GB300 generalized-winding-number library.
 *
 * The library evaluates the generalized winding number (GWN) of an oriented
 * triangle mesh M (open, self-intersecting, non-manifold or a soup) at query
 * points q, by the antipodal method of arXiv 2605.01536:
 *
 *     w(q) = chi(x0) + (1/4pi) * sum_{(a,b) in dM} Area(A, B, x1)        (Eq. 9)
 *
 * with x0 = (0,0,1), x1 = -x0 (Supp. S2.1), chi the signed number of crossings
 * of the ray q + t x0, t > 0, with M (Sec. 3.2: +1 where x0 . n > 0, -1 where
 * x0 . n < 0), dM the oriented boundary edges left after interior edges cancel
 * (Sec. 4.1), A = (a-q)/|a-q|, B = (b-q)/|b-q| and Area the signed spherical
 * triangle area of van Oosterom and Strackee (Sec. 3.3).  The plain direct sum
 * w(q) = (1/4pi) sum_T Area(T) (Sec. 3.1, Eq. 2) is provided as the baseline.
 *
 * Robustness (Supp. S2.1): every query is symbolically perturbed to
 * q + (e1, e2, e3), e3 << e2 << e1, and the crossing predicates and the sign of
 * the area term on the atan2 branch cut are evaluated exactly on the FP32
 * inputs (an FP32 filter first, exact FP64 expansion arithmetic when the filter
 * cannot decide), so that the two discontinuities coincide and w never carries
 * an off-by-integer error.  On the mesh itself w is defined as w(q_eps); on the
 * boundary curve dM it is undefined.
 *
 * Conventions for every call:
 *   - Return value: GWN_OK (0) or one of the GWN_ERR_* codes below; on error
 *     gwn_last_error() returns a message (thread-local, valid until the next
 *     call on the same thread).  Nothing is written to outputs on argument
 *     errors.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Calls whose pointers are all device pointers only
 *     enqueue work on `stream` and return without synchronising, unless the
 *     call's comment says otherwise.
 *   - Pointers: query and output arrays may be device pointers or host
 *     pointers (pageable or pinned).  If any of them is a host pointer the call
 *     stages through temporary device buffers (stream-ordered allocations on
 *     `stream`), copies the results back and synchronises `stream` before
 *     returning.  Caller-owned memory is
 *     never retained after a call returns.
 *   - Layouts: points are float32 [n][3] (x, y, z interleaved, 12 bytes per
 *     point, 4-byte aligned); faces are int32 [nt][3] (counter-clockwise seen
 *     from the side the normal points to); per-query outputs are dense arrays
 *     of length n.
 *   - Mesh handles are opaque and own all of their device memory.  A handle may
 *     be used from several streams concurrently for queries, but
 *     gwn_build_accel and gwn_mesh_destroy must not overlap any other use.
 *   - n = 0 is valid and does nothing.  Coordinates must be finite and of
 *     magnitude below 2^60 (squared distances must stay finite in FP32).
 */
#ifndef GWN_H
#define GWN_H

#include <stdint.h>

#if defined(__GNUC__)
#define GWN_API __attribute__((visibility("default")))
#else
#define GWN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int gwn_status;

enum {
    GWN_OK = 0,
    GWN_ERR_INVALID_ARG = 1,      /* null pointer, negative size, bad config */
    GWN_ERR_INVALID_MESH = 2,     /* face index out of range or non-finite vertex */
    GWN_ERR_NOT_BUILT = 3,        /* gwn_build_accel has not run on this mesh */
    GWN_ERR_CUDA = 4,             /* a CUDA runtime call failed (message says which) */
    GWN_ERR_OOM = 5,              /* device allocation failed */
    GWN_ERR_TRAVERSAL_LIMIT = 6   /* the BVH walk exceeded its node budget (corrupt tree) */
};

typedef struct gwn_mesh gwn_mesh;

/* Tuning knobs; zero-initialise and set what you need (0 = default). */
typedef struct gwn_config {
    int32_t queries_per_thread;   /* boundary-sum kernel: queries held per thread (1,2,4,8) */
    int32_t boundary_tile;        /* boundary points staged in shared memory per step */
    int32_t chain_boundary;       /* 1 (default): share points between consecutive boundary
                                     edges of a loop; -1: store every edge as its own two points */
    float classify_margin;        /* |w - 1/2| at or below which gwn_classify re-evaluates the
                                     boundary sum in FP64 (default 1e-4) */
    int32_t quantize_bits;        /* 0 (default): the perturbed predicates are decided exactly on
                                     the FP32 inputs.  30: as in the paper's Supp. S2.1, inputs are
                                     snapped to a 30-bit fixed-point grid over the mesh's bounding
                                     box (quantum 2^e, the smallest power of two that maps every
                                     vertex into [-2^29, 2^29] around the box centre) and the
                                     crossing test and boundary branch-cut signs are decided on the
                                     snapped integers; results match the default except for
                                     queries within about one quantum of the surface.  Not
                                     supported by the grid entry points. */
    int32_t fp64_cancel;          /* 0 (default) or 1: every boundary term is FP32 except those
                                     whose denominator d = H_a H_b + A_x B_x + A_y B_y (Eq. 9's
                                     van Oosterom-Strackee form with x1 = -z) cancels to below
                                     2^-6 H_a H_b, which are evaluated in FP64 from the FP32
                                     inputs.  Such terms come from boundary edges passing very
                                     close to the query, where FP32 rounding grows like the edge
                                     length over the distance; with them in FP64 no FP32 term is
                                     worse-conditioned than about 65.  Applies to gwn_query_batch,
                                     gwn_classify, gwn_classify_static and the batched launch.
                                     -1: every boundary term in FP32 (the plain form; its error
                                     exceeds 1e-5 within ~1e-4 edge lengths of dense boundaries).
                                     The batched launch always uses the default.  Must be -1, 0
                                     or 1. */
    int32_t group_test;           /* Boundary terms are summed 8 at a time through a complex
                                     product and one atan2 (Eq. 9's angles added as arguments);
                                     a term enters the product only if the product's argument
                                     stays the exact sum.  1: per-term test, each angle below
                                     pi/8.  2: running test, d > 5e-5 and the product keeps a
                                     positive real part (fewer terms on the slower one-by-one
                                     path where many are steep, as on random soups, but 9%
                                     slower where few are).  0 (default): 2 when the boundary
                                     has at least one edge per two triangles, else 1.  Results
                                     agree to rounding either way.  The batched launch always
                                     uses 2.  Must be 0, 1 or 2. */
    int32_t reserved[9];
} gwn_config;

/* Sizes of a mesh after gwn_build_accel. */
typedef struct gwn_mesh_info {
    int64_t nv, nt;               /* vertices and triangles */
    int64_t n_boundary_edges;     /* |dM|, counted with multiplicity */
    int64_t n_boundary_points;    /* points of the chained boundary polylines */
    int64_t n_boundary_loops;     /* closed loops the boundary was chained into */
    int64_t n_bvh_nodes;          /* 2 nt - 1 for nt > 0 */
    int32_t built;                /* 1 after gwn_build_accel */
    int32_t device;               /* CUDA device ordinal the mesh lives on */
} gwn_mesh_info;

/* Event counters accumulated on the device since creation or the last reset. */
typedef struct gwn_counters {
    uint64_t error_flags;         /* bit 0: traversal node budget exceeded */
    uint64_t exact_edge;          /* 2-D edge predicates decided by the exact path */
    uint64_t exact_plane;         /* plane-side predicates decided by the exact path */
    uint64_t exact_branch;        /* branch-cut numerator signs decided by the exact path */
    uint64_t apex_terms;          /* boundary terms taken as the limit for a vertex straight above */
    uint64_t degenerate_terms;    /* boundary terms with numerator = denominator = 0
                                     (query on the boundary curve or a vertical boundary edge) */
    uint64_t fp64_reevaluations;  /* queries re-evaluated in FP64 by gwn_classify */
    uint64_t surrogate_queries;   /* queries gwn_classify put to the learned surrogate */
    uint64_t surrogate_fallbacks; /* of those, queries sent on to the exact path (margin or band) */
    uint64_t gradient_skipped;    /* gradient terms dropped as singular (query on the boundary curve or a
                                     boundary point exactly straight above or below it) */
    uint64_t cancel_terms;        /* boundary terms evaluated in FP64 because their denominator
                                     cancels (gwn_config.fp64_cancel) */
    uint64_t cancel_overflow;     /* cancelling terms beyond a warp's queue in the batched launch
                                     whose query was not listed for FP64 re-evaluation (0 unless a
                                     list could not be kept) */
    uint64_t reserved[4];
} gwn_counters;

/* Library version string. */
GWN_API const char *gwn_version(void);

/* Message for the last error on the calling thread ("" if none). */
GWN_API const char *gwn_last_error(void);

/*
 * Create a mesh from nv vertices V (float32 [nv][3]) and nt faces F
 * (int32 [nt][3]), host or device pointers.  The data are copied; the caller
 * keeps ownership of V and F.  Validates that every index is in [0, nv) and
 * every coordinate is finite (GWN_ERR_INVALID_MESH otherwise); this check
 * synchronises `stream`.  Degenerate triangles are allowed: a triangle whose
 * projection has zero area is never crossed (Supp. S2.1).  The mesh lives on the
 * current CUDA device.  cfg may be NULL.  Paper: the inputs p, M of Algorithm 1.
 */
GWN_API gwn_status gwn_mesh_create(const float *V, int64_t nv, const int32_t *F, int64_t nt,
                           const gwn_config *cfg, void *stream, gwn_mesh **out);

/* Free a mesh and all of its device memory (synchronises the device first). */
GWN_API gwn_status gwn_mesh_destroy(gwn_mesh *mesh);

/*
 * Build the acceleration data: the oriented boundary dM (Sec. 4.1: each
 * undirected edge {u,v} of net multiplicity m = #(u->v) - #(v->u) appears |m|
 * times in its net direction; vertices are matched by index, not welded by
 * position), its chaining into closed loops, and a linear BVH over the
 * triangles (Morton codes of centroids, radix sort, Karras hierarchy, bottom-up
 * box refit, escape links for stackless traversal).  Replaces the paper's
 * Embree BVH (Sec. 5).  Idempotent.  Synchronises `stream` once to read the
 * boundary size.
 */
GWN_API gwn_status gwn_build_accel(gwn_mesh *mesh, void *stream);

/* Sizes of the mesh (host call, no synchronisation). */
GWN_API gwn_status gwn_mesh_get_info(const gwn_mesh *mesh, gwn_mesh_info *info);

/*
 * Copy the oriented boundary edges into edges (int32 [cap][2], host or device),
 * sorted by the undirected key (min(u,v), max(u,v)); *n_out receives |dM|.
 * Fails with GWN_ERR_INVALID_ARG if cap < |dM|.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_mesh_get_boundary(const gwn_mesh *mesh, int32_t *edges, int64_t cap,
                                 int64_t *n_out, void *stream);

/*
 * Copy the chained boundary points the query kernels stream (float32
 * [cap][4]: x, y, z, flag; flag 1 = an edge runs from this point to the next
 * one), host or device; *n_out receives their number.  Each closed loop of dM
 * is stored as its vertices followed by its first vertex again (flag 0).
 * Fails with GWN_ERR_INVALID_ARG if cap is too small.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_mesh_get_boundary_points(const gwn_mesh *mesh, float *points, int64_t cap,
                                                int64_t *n_out, void *stream);

/*
 * Antipodal GWN (Eq. 9, Algorithm 1 with x0 = +z) of n query points q
 * (float32 [n][3]).  Writes w (float32 [n]) and, if chi is not NULL, the exact
 * signed crossing number chi (int32 [n]).  Requires gwn_build_accel
 * (GWN_ERR_NOT_BUILT).  w is accurate to about 1e-6 absolute for FP32 inputs
 * (FP32 terms, FP64 accumulation per query).
 */
GWN_API gwn_status gwn_query_batch(const gwn_mesh *mesh, const float *q, int64_t n, float *w,
                           int32_t *chi, void *stream);

/*
 * Only the signed crossing number chi (int32 [n]) of the ray q + t(0,0,1)
 * (Sec. 3.2), exact under the perturbation of Supp. S2.1.  For a closed mesh
 * this is the winding number itself (Sec. 4.1).  Requires gwn_build_accel.
 */
GWN_API gwn_status gwn_query_chi(const gwn_mesh *mesh, const float *q, int64_t n, int32_t *chi,
                         void *stream);

/*
 * Direct solid-angle sum w = (1/4pi) sum_T Area(T) (Sec. 3.1, Eq. 2) with the
 * unnormalised van Oosterom-Strackee area per triangle (Sec. 3.3): the
 * baseline the antipodal method is compared against (Sec. 5.1).  Does not need
 * gwn_build_accel.  Undefined (may be NaN) for queries on the surface.
 */
GWN_API gwn_status gwn_query_direct(const gwn_mesh *mesh, const float *q, int64_t n, float *w,
                            void *stream);

/*
 * Gradient of w with respect to the query point (Supp. S4, Algorithm 3 with
 * x0 = +z): grad[3 i + k] = d w / d q_k at q_i (float32 [n][3], row-major).  The
 * crossing count is piecewise constant, so only the boundary terms contribute
 * (a closed mesh gives 0).  FP32 terms, FP64 accumulation.  A term that is
 * singular (q on the boundary curve, or a boundary point exactly straight
 * above or below q) is dropped and counted in gwn_counters.gradient_skipped;
 * the gradient is undefined on dM.  Requires gwn_build_accel.
 */
GWN_API gwn_status gwn_query_gradient(const gwn_mesh *mesh, const float *q, int64_t n, float *grad,
                                      void *stream);

/*
 * gwn_query_chi, instrumented: the same crossing counts (exact-predicate
 * meshes only) plus, summed over the n queries, the BVH nodes the walks read
 * (*nodes_out) and the triangles they tested (*triangles_out) -- the counts
 * behind the traversal's algorithmic bytes (nodes x 32 B + triangles x 36 B +
 * 12 B + 4 B per query).  A separate kernel, so the timed path carries no
 * counting.  Synchronises `stream`.  GWN_ERR_INVALID_ARG for a fixed-point mesh.
 */
GWN_API gwn_status gwn_query_chi_visits(const gwn_mesh *mesh, const float *q, int64_t n, int32_t *chi,
                                        uint64_t *nodes_out, uint64_t *triangles_out, void *stream);

/*
 * Rectilinear grids with ray reuse (Supp. S3).  The grid's cells are the points
 * (x[i], y[j], z[k]) for i < nx, j < ny, k < nz; outputs are indexed
 * [(k * ny + j) * nx + i] (x fastest).  x, y, z are float32 arrays in host or
 * device memory (copied by the call); z must be non-decreasing; all
 * coordinates finite; nx * ny * nz <= 2^31 - 1.  One BVH walk per (x, y)
 * column replaces nz walks; each cell's crossing decision is the same exact,
 * perturbed predicate the per-query path evaluates at that point, so chi is
 * bit-identical to gwn_query_chi on the same points.  Both calls synchronise
 * `stream` once and require gwn_build_accel.
 */
GWN_API gwn_status gwn_query_grid_chi(const gwn_mesh *mesh, const float *x, int32_t nx, const float *y, int32_t ny,
                                      const float *z, int32_t nz, int32_t *chi, void *stream);

/* Labels (and w when w_or_null is not NULL) of every grid cell: chi by ray
 * reuse, then the boundary sum and FP64 re-evaluation as in gwn_classify (a
 * closed mesh needs neither: w = chi). */
GWN_API gwn_status gwn_classify_grid(const gwn_mesh *mesh, const float *x, int32_t nx, const float *y, int32_t ny,
                                     const float *z, int32_t nz, uint8_t *label, float *w_or_null, void *stream);

/*
 * Inside/outside labels: label[i] = 1 iff w(q_i) > 1/2 (uint8 [n]); w_or_null
 * receives w when not NULL.  Computed by the antipodal method; a query whose
 * FP32 w lies within cfg.classify_margin of 1/2 has its boundary sum
 * re-evaluated in FP64 before labelling (Sec. 5.2 reports FP32 as accurate to
 * the type's limit; the margin turns that into exact labels).  Requires
 * gwn_build_accel.
 */
GWN_API gwn_status gwn_classify(const gwn_mesh *mesh, const float *q, int64_t n, uint8_t *label,
                        float *w_or_null, void *stream);

/*
 * Copy (and, if reset != 0, zero) the mesh's device event counters.
 * Synchronises `stream`.  Returns GWN_ERR_TRAVERSAL_LIMIT if the traversal
 * error flag is set.
 */
GWN_API gwn_status gwn_get_counters(gwn_mesh *mesh, gwn_counters *out, int reset, void *stream);

/*
 * gwn_classify without any device allocation (the paper has no counterpart; a
 * library addition).  For callers that cannot allocate device memory on the
 * call path: hosts that reserve their whole device-memory budget up front (a
 * fixed pool, or another framework's allocator owning the GPU) and
 * latency-critical loops that must stay out of the CUDA allocator, which can
 * take locks, synchronise or grow a pool.  It always runs the exact path
 * (crossing count, boundary sum, FP64 re-evaluation near 1/2): an attached
 * learned surrogate is not used.  Its labels are the exact ones, and w is
 * bit-identical to gwn_classify's on a mesh without a surrogate (each query's
 * arithmetic does not depend on the rest of the batch or its order).
 *   - Scratch: one 32 MiB file-scope device array per GPU that loads the
 *     library, held until the process exits; every call uses it.
 *   - Limit: n <= 2,097,152 queries per call; larger n fails with
 *     GWN_ERR_INVALID_ARG.  q, label and w_or_null must be device memory of
 *     the mesh's GPU (GWN_ERR_INVALID_ARG otherwise, with nothing launched).
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Calls that overlap on the GPU (different streams, or different threads
 *     without ordering) race on the shared array and give wrong results: order
 *     them.  The array keeps the last call's contents; the call clears the
 *     counter it needs.
 */
GWN_API gwn_status gwn_classify_static(const gwn_mesh *mesh, const float *q, int64_t n, uint8_t *label,
                                       float *w_or_null, void *stream);

/* ------------------------------------------------------------------------
 * Batches: many meshes with uneven query sets in one persistent launch.
 * (Not in the paper, which evaluates one mesh at a time; its parallelism is
 * over queries, Sec. 5.)
 * ------------------------------------------------------------------------ */
typedef struct gwn_batch gwn_batch;

/* Schedule of a batch; zero-initialise for defaults or let gwn_batch_autotune pick. */
typedef struct gwn_batch_config {
    int32_t queries_per_thread;   /* 2 or 4 (default 4): queries per work item = 256 x this */
    int32_t points_per_item;      /* boundary points per work item (default 8192) */
    int32_t tile;                 /* boundary points staged in shared memory (default 512) */
    int32_t grid_blocks;          /* persistent blocks (default: resident blocks per SM x SMs) */
    int32_t use_graph;            /* >= 0 (default): capture and replay a CUDA graph; -1: plain launches */
    int32_t tune_queries_per_mesh;/* gwn_batch_autotune times candidates on at most this many queries
                                     of each mesh (default 16384) */
    int32_t reserved[10];
} gwn_batch_config;

/*
 * Create a batch over n_mesh built meshes (all on one device).  Queries of
 * mesh i are rows q_offsets[i] .. q_offsets[i+1]-1 of the concatenated query
 * array given to gwn_batch_run (q_offsets: host int64 [n_mesh + 1], q_offsets[0]
 * = 0, non-decreasing).  The meshes must outlive the batch.  Synchronous.
 */
GWN_API gwn_status gwn_batch_create(const gwn_mesh *const *meshes, int32_t n_mesh, const int64_t *q_offsets,
                                    const gwn_batch_config *cfg, gwn_batch **out);
GWN_API gwn_status gwn_batch_destroy(gwn_batch *batch);

/*
 * Antipodal w (float32 [total]) and, if chi is not NULL, chi (int32 [total])
 * for every query of the batch, in one persistent launch over a work queue
 * sorted by cost.  Device pointers only.  The launch sequence is captured into
 * a CUDA graph on a stream the batch owns, ordered after the work already
 * queued on `stream` and before anything queued on it later; the graph is
 * reused while (q, w, chi) stay the same.  The FP64 accumulation order of a
 * query's boundary chunks is not fixed (atomic adds): w is reproducible to
 * FP64 rounding, not bitwise.  Runs of one batch must not overlap.
 */
GWN_API gwn_status gwn_batch_run(gwn_batch *batch, const float *q, float *w, int32_t *chi, void *stream);

/*
 * Time candidate schedules (queries per item 2 or 4, points per item 2048,
 * 8192 or 32768, one or two grids' worth of resident blocks) on this batch's
 * meshes with the first cfg.tune_queries_per_mesh queries of each, keep the
 * fastest, and record it in cache_path (one JSON object per
 * line, keyed by the batch's size class; NULL = no cache).  A cached entry for
 * the key is applied without timing.  Writes w; synchronises `stream`.
 */
GWN_API gwn_status gwn_batch_autotune(gwn_batch *batch, const float *q, float *w, void *stream,
                                      const char *cache_path, gwn_batch_config *chosen);

/* The schedule in use and the number of work items. */
GWN_API gwn_status gwn_batch_get_config(const gwn_batch *batch, gwn_batch_config *cfg, int64_t *n_items);

/*
 * Tensor-core self-test (library diagnostics, no paper counterpart):
 * C[128][64] = A[128][K] x B[64][K]^T with A, B row-major BF16 device arrays
 * and C an FP32 device array, K = 64 or 128, computed by one tcgen05 MMA chain
 * into TMEM.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_debug_tc_gemm(const void *A, const void *B, int32_t K, float *C, void *stream);

/* ------------------------------------------------------------------------
 * Learned surrogate (not in the paper; its future-work item of a fast
 * approximation of the fractional part).  A per-mesh MLP of w: Fourier
 * features (the sample box mapped to [-1,1]^3; x, y, z and sin, cos of
 * pi 2^(7k/15) x_d for k < 16), four 64-wide ReLU layers, a linear output;
 * trained with mean squared error and Adam on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulators).  Once trained, gwn_classify answers a query
 * with the network where |w_hat - 1/2| > margin and the query lies outside the
 * surface band (the cells of a grid over the box that a triangle's bounding
 * box touches, dilated: there w jumps and a smooth network is unreliable), and
 * with the exact antipodal path (including its FP64 re-evaluation) everywhere
 * else; it then synchronises `stream` once to size the exact pass.
 * ------------------------------------------------------------------------ */
typedef struct gwn_mlp_config {
    int32_t steps;                /* Adam steps (default 3000) */
    int32_t batch;                /* samples per step (default 16384) */
    float lr;                     /* learning rate (default 1e-3) */
    float margin;                 /* gate half-width around 1/2 (default 0.1) */
    uint64_t seed;                /* initial weights and batch sampling (counter-based) */
    float beta1, beta2, eps;      /* Adam (defaults 0.9, 0.999, 1e-8) */
    int32_t band_res;             /* surface band grid: cells per axis over the box (default 256, max 1024;
                                     negative: no band) */
    int32_t band_dilate;          /* band dilation in cells (default 1; negative: none) */
    float chi_tol;                /* gate: the network answers only where its w lies within chi_tol of
                                     the exact crossing count chi (computed for every query; with it
                                     an answered label is [chi >= 1], wrong only where the boundary
                                     term exceeds 1/2 in magnitude) (default 0.25; negative: no test) */
    int32_t reserved[6];
} gwn_mlp_config;

/* Number of FP32 parameters of the network (20801). */
GWN_API int32_t gwn_surrogate_num_params(void);

/*
 * Train the mesh's surrogate from scratch on n samples (device float32
 * [n][3]) with targets (device float32 [n]) or, when targets is NULL, w from
 * this library's antipodal path (needs gwn_build_accel).  The input box is the
 * samples' bounding box.  final_loss (host, may be NULL) receives the last
 * batch's mean squared error.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_surrogate_train(gwn_mesh *mesh, const float *samples, const float *targets, int64_t n,
                                       const gwn_mlp_config *cfg, float *final_loss, void *stream);

/* The network's raw output w_hat (device float32 [n]) for device queries q. */
GWN_API gwn_status gwn_surrogate_predict(const gwn_mesh *mesh, const float *q, int64_t n, float *w_hat,
                                         void *stream);

/*
 * Get (set = 0) or set (set = 1) the FP32 parameters (host array of
 * gwn_surrogate_num_params() floats: W1 [64][128], b1, W2, b2, W3, b3, W4, b4
 * [64][64] / [64], w5 [64], b5) and the input box (host float [6]: lo xyz,
 * hi xyz; may be NULL).  Setting marks the surrogate as trained.
 */
GWN_API gwn_status gwn_surrogate_params(gwn_mesh *mesh, float *params, float *box, int32_t set);

/*
 * Gradient of the mean squared error over n samples (device q [n][3], device
 * targets [n]) with respect to the parameters, on the same kernels training
 * uses; written to grad (host, gwn_surrogate_num_params() floats), the loss to
 * *loss (host, may be NULL).  n <= 2^22.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_surrogate_grad(gwn_mesh *mesh, const float *q, const float *targets, int64_t n, float *grad,
                                      float *loss, void *stream);

/*
 * Calibrate the gate on held-out samples (device float32 [n][3], n < 2^31,
 * drawn like the queries to be classified): the exact path labels them, and the
 * margin becomes the smallest value >= min_margin (in steps of 1/2048) at which
 * at most floor(max_error_rate * n) samples have |w_hat - 1/2| > margin and a
 * label that differs from the exact one.  *margin_out (host, may be NULL)
 * receives it, *errors_at_margin (host, may be NULL) that count.  The margin
 * is stored with the surrogate and used by gwn_classify.  Synchronises `stream`.
 */
GWN_API gwn_status gwn_surrogate_calibrate(gwn_mesh *mesh, const float *samples, int64_t n, double max_error_rate,
                                           float min_margin, float *margin_out, int64_t *errors_at_margin,
                                           void *stream);

/* Save / load the surrogate (parameters, Adam moments, step count, box, config). */
GWN_API gwn_status gwn_surrogate_save(const gwn_mesh *mesh, const char *path);
GWN_API gwn_status gwn_surrogate_load(gwn_mesh *mesh, const char *path);

/* Drop the surrogate; gwn_classify is exact again. */
GWN_API gwn_status gwn_surrogate_detach(gwn_mesh *mesh);

/* ------------------------------------------------------------------------
 * Parametric surfaces (Sec. 4.4, Algorithm 2): untrimmed bicubic Bezier
 * patches, w = chi + the sum over the boundary curves of the integral of
 * Algorithm 2's f(phi, t), with x0 = +z.
 *   chi: each patch is subdivided down to bilinear patches within flat_tol of
 *     the surface (Sec. 4.4.1's tau), then met by the +z ray in closed form;
 *     a crossing found from both sides of a seam counts once.  Closer to the
 *     surface than that tolerance the crossing count may be off by one (the
 *     paper re-casts such rays; results there are not meaningful anyway).
 *   the integrals: adaptive Gauss-Kronrod 15 per curve (Sec. 4.4 uses GK15).
 *     Default: panels evaluated in FP32 from a per-curve tree of panels whose
 *     control points are stored relative to each panel's centre (errors of
 *     the panel's own scale), FP64 below depth 12; fp64 = 1 evaluates every
 *     panel in FP64.  Error: about quad_tol per curve plus, with FP32
 *     panels, at most about 2^-19 times the sum over the curves of the
 *     integral of (|r_x dr_y| + |r_y dr_x|) g / 4pi >= the integral of |f|
 *     (an FP32 panel is accepted at the latest at 2^-20 of its own such
 *     integral, the FP32 rounding level of its 15 values, and only while that
 *     level is below 2^-18 / 4pi; beyond it the panel is refined, in FP64
 *     below depth 12).
 * ------------------------------------------------------------------------ */
typedef struct gwn_param gwn_param;

typedef struct gwn_param_config {
    double quad_tol;      /* error target per curve, per unit of parameter length (default 1e-10) */
    double flat_tol;      /* bilinear tolerance relative to the control points' extent (default 1e-6) */
    int32_t fp64;         /* 1: every quadrature panel in FP64; 0 (default): FP32 panels, see above */
    int32_t max_panels;   /* quadrature panel budget of a query: max_panels per curve (default 1024) */
    int32_t max_nodes;    /* subdivision node budget of a ray: max_nodes per patch (default 65536) */
} gwn_param_config;

/* Fill *cfg with the defaults above. */
GWN_API void gwn_param_config_default(gwn_param_config *cfg);

/*
 * patches: float32 [np][4][4][3] (host or device, copied), control point (i, j)
 * of patch p at [p][i][j], i along u, j along v; the surface is oriented by
 * S_u x S_v.  The boundary of the union is extracted here: each patch's four
 * edge curves run counter-clockwise about its normal, and a curve cancels
 * against its exact reverse (a shared edge of consistently oriented patches,
 * the identification of Sec. 5's parametric comparison).  cfg may be NULL
 * (defaults).  Non-finite control points: GWN_ERR_INVALID_MESH.  Synchronous.
 */
GWN_API gwn_status gwn_param_create(const float *patches, int32_t np, const gwn_param_config *cfg,
                                    gwn_param **out);
GWN_API gwn_status gwn_param_destroy(gwn_param *surface);

/* Boundary curves of the union (host float32 [cap][4][3]); *n_out = their count. */
GWN_API gwn_status gwn_param_get_boundary(const gwn_param *surface, float *curves, int32_t cap, int32_t *n_out);

/*
 * w (float32 [n]) and optionally chi (int32 [n]) of n queries q (float32
 * [n][3]); device pointers only (GWN_ERR_INVALID_ARG otherwise).
 * Asynchronous on `stream`.
 */
GWN_API gwn_status gwn_param_query(const gwn_param *surface, const float *q, int64_t n, float *w,
                                   int32_t *chi_or_null, void *stream);

/*
 * w and optionally chi of every cell (x[i], y[j], z[k]) of a grid, indexed
 * [(k * ny + j) * nx + i]; x, y, z host or device float32 (copied), z finite
 * and non-decreasing (else GWN_ERR_INVALID_ARG), w and chi device pointers.
 * One ray per (x, y) column serves all its cells (the ray reuse Sec. 4.4.1
 * applies to voxelization): each crossing adds its sign below it, a suffix
 * sum over the column gives every cell its count; the boundary integrals are
 * evaluated per cell.  z is validated on the host (read in place, or copied
 * back synchronously from device memory); the kernels run asynchronously on
 * `stream`.
 */
GWN_API gwn_status gwn_param_query_grid(const gwn_param *surface, const float *x, int32_t nx, const float *y,
                                        int32_t ny, const float *z, int32_t nz, float *w, int32_t *chi_or_null,
                                        void *stream);

/* Since the last reset: queries (or grid columns) whose subdivision hit its
 * depth, stack, node or hit budget; points whose boundary integral ended above
 * its error target; quadrature panels evaluated (each 15 integrand values) and
 * how many of them in FP64.  Any pointer may be NULL.  Synchronous. */
GWN_API gwn_status gwn_param_status(const gwn_param *surface, uint64_t *budget_hits, uint64_t *unconverged,
                                    uint64_t *panels, uint64_t *panels_fp64, int reset);

/* Per-kernel timing record filled by gwn_profile_read. */
typedef struct gwn_kernel_stat {
    char name[32];                /* step name, e.g. "boundary_sum" */
    int64_t launches;             /* times the step ran since profiling was enabled or last read */
    double total_ms;              /* summed device time between CUDA events recorded on
                                     the launching stream around each run of the step */
    int64_t kernels;              /* CUDA kernels those runs launched */
} gwn_kernel_stat;

/*
 * Enable (on != 0) or disable per-kernel timing for all meshes in the process.
 * While enabled, every kernel launch of the query and build paths is bracketed
 * by two CUDA events on its stream.  Enabling clears earlier records.
 * Instrumentation only; not part of the paper's method.
 */
GWN_API gwn_status gwn_profile_enable(int on);

/*
 * Synchronise on the recorded events, aggregate them per kernel name into
 * stats (host array of cap entries; *n_out receives the number of kernel names,
 * which may exceed cap) and clear the records.
 */
GWN_API gwn_status gwn_profile_read(gwn_kernel_stat *stats, int cap, int *n_out);

/*
 * Measured pipe throughputs of the current device behind the ALU rooflines
 * (instrumentation, not part of the paper's method): *ffma_per_s = scalar FP32
 * FMA thread-instructions per second, *ffma2_per_s = paired FP32 FMA
 * thread-instructions per second (each is two FMAs, the form the boundary
 * kernels use), *mufu_per_s = SFU reciprocal / reciprocal-square-root
 * thread-operations per second; from independent dependency chains on every SM
 * timed with CUDA events (best of 3 runs after a warm-up); *sm_count = SMs.
 * Takes about 0.3 s; synchronises.
 */
GWN_API gwn_status gwn_measure_pipe_peaks(double *ffma_per_s, double *ffma2_per_s, double *mufu_per_s,
                                          int32_t *sm_count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GWN_H */
