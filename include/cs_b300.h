/*
 * cs_b300.h -- C ABI of the B300 engine for the CollisionSplatting
 * conservative collision metric (arXiv 2609.35619).
 *
 * The engine evaluates, for a batch of posed robot primitives (spheres or
 * ellipsoids) and every Gaussian of a resident 3DGS scene, the conservative
 * scaling-function metric of Section II-B and reduces it per primitive to the
 * quantities the planners of Sections II-D and II-E consume:
 *
 *   Eq. 2   Sigma_i = R(q_i) diag(s_i)^2 R(q_i)^T
 *   Eq. 5   s^2_ij  = (mu_i - c_j)^T A_j (mu_i - c_j)
 *   Eq. 6   A_j     = R_j diag(1/a^2, 1/b^2, 1/c^2) R_j^T   (sphere: I / r^2)
 *   Eq. 7   sigma^2_ij = g Sigma_i g^T,  g = 2 A_j (mu_i - c_j)
 *   Eq. 8   st^2_ij = max(0, s^2_ij - n_sigma sqrt(sigma^2_ij))
 *   Eq. 11  dc_ij   = d_max exp(-gamma max(st^2_ij - s_min, 0))
 *
 * Reductions over the neighbour set N_j = { i : st^2_ij <= S_cut },
 * S_cut = s_min + ln(1/eps)/gamma (every omitted cost term is below
 * eps * d_max):
 *   mean cost  = sum_{N_j} dc / |N_j|   (0 when N_j is empty; Section II-D)
 *   sum cost   = sum_{N_j} dc
 *   min st^2   over N_j                  (+inf when empty)
 *   softmin    = -tau ln sum_{N_j} exp(-st^2/tau)   (+inf when empty;
 *                the recursive softmin of Section II-B, computed online)
 *   collide    = #{ i in N_j : st^2 < 1 } > k_thr   (Section II-E)
 *
 * Conventions common to every entry point:
 *   - float32 everywhere; quaternions are (w, x, y, z) and are normalised by
 *     the library; scales are per-axis standard deviations.
 *   - Device pointers are CUDA global-memory pointers of the current device
 *     (e.g. from torch tensors); "host" pointers are ordinary CPU memory
 *     (pinned memory gives asynchronous copies).  The caller owns every
 *     buffer it passes; the library owns the scene and its scratch memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     enqueued asynchronously unless stated otherwise.  Argument errors are
 *     returned synchronously, before anything is enqueued.
 *   - Device-side conditions (invalid query rows, a bounded wait that ran
 *     out) are recorded in a per-stream error word and reported by cs_sync.
 *   - Query scratch (sort keys, prepared rows, host staging) is pooled per
 *     (device, stream) and reused; calls on the same stream share it, calls
 *     on different streams may run concurrently.
 *   - cs_last_error() returns a thread-local message for the last failure.
 */
#ifndef CS_B300_H
#define CS_B300_H

#include <stdint.h>

#if defined(__GNUC__)
#define CS_API __attribute__((visibility("default")))
#else
#define CS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_scene cs_scene; /* opaque, library-owned, device-resident */

typedef enum cs_status {
    CS_OK = 0,
    CS_ERR_INVALID_ARG = -1, /* bad pointer, size, parameter or input value */
    CS_ERR_NO_MEMORY = -2,   /* a device allocation failed */
    CS_ERR_CUDA = -3,        /* a CUDA runtime call failed (message in cs_last_error) */
    CS_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out */
    CS_ERR_BAD_HANDLE = -5,  /* NULL or destroyed scene handle */
    CS_ERR_UNSUPPORTED = -6, /* valid request the library does not implement */
    CS_ERR_BOUNDS = -7       /* a device-side index check failed (builds compiled with
                                CS_DEBUG only): the access was skipped or redirected to an
                                in-range element, no trap; the call's outputs are not valid */
} cs_status;

typedef enum cs_prim_type {
    CS_PRIM_SPHERE = 0,    /* 4 floats per row: cx, cy, cz, r            (Eq. 6, a=b=c=r) */
    CS_PRIM_ELLIPSOID = 1  /* 10 floats per row: cx, cy, cz, qw, qx, qy, qz, a, b, c (Eq. 6) */
} cs_prim_type;

typedef enum cs_metric_mode {
    CS_METRIC_MEAN_COST = 0,  /* Eq. 11 averaged over N_j (MPPI, Section II-D) */
    CS_METRIC_SUM_COST = 1,   /* Eq. 11 summed over N_j */
    CS_METRIC_MIN_S2 = 2,     /* min over N_j of Eq. 8 */
    CS_METRIC_SOFTMIN_S2 = 3, /* softmin over N_j of Eq. 8 (Section II-B) */
    CS_METRIC_FLAGS = 4       /* collision flags only (Section II-E), with early exit: a row
                                 stops once its in-collision count exceeds k_thr, and with
                                 group_size > 0 the rows of a group stop once one of them
                                 collides.  out_collide per row: 1 in collision, 0 free,
                                 2 not finished because its group collides; the group flag
                                 is exact.  out_metric, out_count, out_group_metric are not
                                 written; cs_query_grad rejects this mode. */
} cs_metric_mode;

/* Scene description for cs_scene_create (Section II-A, Eq. 1-2). */
typedef struct cs_scene_desc {
    int64_t n;              /* number of Gaussians, >= 0 */
    const float *means;     /* [n,3] Gaussian means (world frame) */
    const float *scales;    /* [n,3] per-axis standard deviations, >= 0 (a zero axis is a 2DGS disk) */
    const float *quats;     /* [n,4] rotations (w,x,y,z); need not be normalised; 0 -> identity */
    const float *opacity;   /* [n] opacities in [0,1], or NULL (no floater filter) */
    int32_t on_device;      /* 1: the arrays above are device pointers; 0: host pointers */
    int32_t use_filter;     /* floater filter of Section II-C: drop a Gaussian when
                               opacity < opacity_min AND max(scale) > extent_max */
    float opacity_min;      /* default 0.05 */
    float extent_max;       /* default 0.1 (scene units) */
    float cell_size;        /* extent limit of a chunk (up to 32 Gaussians consecutive in
                               Hilbert-curve order); 0 = automatic: twice the edge of a box that
                               holds 32 Gaussians at the mean density of the scene box */
    float tier_quantile;    /* Gaussians whose largest scale exceeds this quantile go to
                               the separately culled large tier; 0 = default 0.99 */
} cs_scene_desc;

#define CS_TILE_TUNED (-1)

/* Per-call parameters for cs_query / cs_query_grad.  Initialise with
 * cs_params_init; every pointer member may be NULL. */
typedef struct cs_params {
    float gamma;               /* Eq. 11 decay, > 0 (default 5) */
    float d_max;               /* Eq. 11 maximum cost per splat (default 1) */
    float s_min;               /* Eq. 11 minimum scaling factor (default 1) */
    float eps;                 /* neighbour-set truncation, 0 < eps < 1 (default 1e-6) */
    float tau;                 /* softmin temperature, > 0 (default 0.05) */
    int32_t k_thr;             /* collide iff the in-collision count exceeds k_thr (default 0) */
    int32_t mode;              /* cs_metric_mode written to out_metric (default mean cost) */
    int32_t group_size;        /* > 0: also reduce runs of group_size consecutive rows
                                  (sum of the metric, OR of the flag; the last run may be
                                  shorter) into out_group_metric / out_group_collide */
    int32_t host_io;           /* 1: prims, nsigma_per_query, grad_out and every output are
                                  host pointers; the call copies in, computes, copies out and
                                  returns after the stream has finished */
    int32_t tile_config;       /* 0 = the default shape (23 for up to 2^17 rows, else 18);
                                  CS_TILE_TUNED = the shape cs_autotune
                                  chose for this scene, primitive type, mode and batch-size
                                  class (the default when none was tuned); otherwise a value
                                  from cs_tile_configs.  cs_query_grad has its own shapes:
                                  1..4 select one, any other value the default */
    const float *nsigma_per_query; /* [Q] n_sigma per row (overrides the scalar), each >= 0 */
    void *stream;              /* cudaStream_t */
    int32_t *out_count;        /* [Q] |N_j| per row */
    float *out_group_metric;   /* [ceil(Q/group_size)] */
    uint8_t *out_group_collide;/* [ceil(Q/group_size)] */
    unsigned long long *out_pair_stats; /* device [2], accumulated (not cleared):
                                  [0] += (query, Gaussian) pairs evaluated after the cull,
                                  [1] += pairs in the neighbour sets (sum of |N_j|) */
    void *eval_events[2];      /* optional cudaEvent_t pair recorded on `stream` immediately
                                  before and after the fused cull+evaluate kernel (tracing) */
    unsigned long long *out_kernel_stats; /* optional device [16], accumulated (not cleared),
                                  counters of the fused kernel (tuning):
                                  [0] stages consumed by consumer warps,
                                  [1] staged chunks tested by consumer warps,
                                  [2] chunks passing a consumer warp's box test,
                                  [3] (primitive, chunk) hits evaluated,
                                  [4] chunks staged by producers,
                                  [5] stages filled by producers,
                                  [6] polls of consumer waits, [7] polls of producer waits,
                                  [8] consumer-warp cycles in total, [9] of which waiting,
                                  [10] producer-warp cycles in total, [11] of which waiting,
                                  [12] consumer cycles until the first stage was ready,
                                  [13] producer cycles until the first stage was closed,
                                  [14] consumer cycles after the last stage (reductions),
                                  [15] tiles */
    int32_t exact_variance;    /* 1: sigma^2 of Eq. 8 is the exact variance of the quadratic
                                  form of Eq. 5 under the Gaussian, 4 d^T A Sigma A d +
                                  2 tr((A Sigma)^2), instead of Eq. 7's first-order term
                                  (more conservative: st^2 can only drop).  The forward call
                                  then runs the default tile shape of its batch size and the
                                  adjoint its default shape (tile_config is ignored).
                                  Default 0. */
    int32_t sweep_count;       /* >= 2: a conservatism sweep in one launch.  cs_query then
                                  evaluates each of the Q rows at every n_sigma of
                                  sweep_nsigma[0 .. sweep_count) (conservatism and
                                  nsigma_per_query are unused) and writes S = sweep_count
                                  blocks: out_metric, out_collide, out_count [S*Q] with row
                                  s*Q + j for value s; group outputs [S*ceil(Q/G)], groups
                                  formed within each block.  Every value gives the same bits
                                  as its own cs_query call.  Not for cs_query_grad, the
                                  flags mode or host_io.  0 or 1 = no sweep (default). */
    float sweep_nsigma[8];     /* the sweep's n_sigma values, each finite and >= 0 */
} cs_params;

/* Scene information returned by cs_scene_info. */
typedef struct cs_scene_info {
    int64_t n_input;      /* Gaussians passed in */
    int64_t n_kept;       /* after the floater filter and input validation */
    int64_t n_grid;       /* kept Gaussians in the main tier */
    int64_t n_large;      /* kept Gaussians in the large tier */
    int64_t n_invalid;    /* rows with non-finite values or negative scales (dropped) */
    int32_t dims[3];      /* nodes of the three levels of the chunk tree (each node
                             bounds 32 chunks or 32 nodes of the level below) */
    float cell_size;      /* extent limit of a chunk of the main tier */
    float sigma_tier;     /* largest scale in the main tier */
    float lo[3], hi[3];   /* bounding box of the kept means */
    int64_t device_bytes; /* device memory held by the scene (without query scratch) */
} cs_scene_info;

/* Fill *p with the defaults listed in cs_params.  Returns CS_ERR_INVALID_ARG
 * for p == NULL. */
CS_API cs_status cs_params_init(cs_params *p);

/* Build a resident scene (Eq. 2 repack, floater filter, Hilbert-ordered
 * chunks of the main and large tiers, the chunk tree) on the current device.
 * Synchronises `stream` a few times (the layout depends on the scene's extent
 * and on the chunk count).  On success *out owns device memory
 * until cs_scene_destroy.  n == 0 gives an empty scene (every query returns
 * an empty neighbour set). */
CS_API cs_status cs_scene_create(const cs_scene_desc *desc, void *stream, cs_scene **out);

/* Release a scene.  The caller must ensure no work using the scene is still
 * running.  NULL is a no-op.  (Query scratch is pooled per stream, not per
 * scene: see cs_release_scratch.) */
CS_API cs_status cs_scene_destroy(cs_scene *scene);

CS_API cs_status cs_scene_info_get(const cs_scene *scene, cs_scene_info *info);

/* Copy the repacked, Hilbert-sorted scene to caller device buffers (any may be
 * NULL): pos [n_kept,4] = (mu, max scale); cov [n_kept,8] = (Sxx, Syy, Szz,
 * 2Sxy, 2Sxz, 2Syz, 0, 0); index [n_kept] = input row of each entry. */
CS_API cs_status cs_scene_export(const cs_scene *scene, float *pos, float *cov, int32_t *index,
                          void *stream);

/* Checkpoint of a built scene (resume without a rebuild).  cs_scene_save
 * writes the scene -- its counts and layout parameters, its one device
 * allocation byte for byte (chunk blocks, chunk tree, export arrays) and the
 * appearance of cs_scene_set_appearance when set -- to the host file `path`
 * (created or truncated), copying on `stream` and synchronising it.  The
 * scene must live on the current device.  Tile shapes chosen by cs_autotune
 * are not saved.  The file is in this library's format (host byte order,
 * format version 1), not portable across byte orders.
 * cs_scene_load reads such a file into a new scene on the current device
 * (*out, owned by the caller until cs_scene_destroy), uploading on `stream`
 * and synchronising it.  A loaded scene answers every query exactly as the
 * saved one did (same layout, same bits).  Errors: CS_ERR_INVALID_ARG for an
 * empty path, a file that cannot be opened, read or written, a wrong magic or
 * format version, a truncated file or a layout that is not self-consistent
 * (region bounds, tree level sizes, slot indices out of range);
 * CS_ERR_NO_MEMORY when the device allocation fails.  *out is NULL on error. */
CS_API cs_status cs_scene_save(const cs_scene *scene, const char *path, void *stream);
CS_API cs_status cs_scene_load(const char *path, void *stream, cs_scene **out);

/* The metric for Q primitives (rows of `prims`, layout per cs_prim_type)
 * against the scene, with conservatism n_sigma = `conservatism` (Eq. 8, >= 0)
 * unless params->nsigma_per_query is given.
 *   out_metric  [Q] float : the params->mode reduction per row (may be NULL
 *                           only when a group output is requested)
 *   out_collide [Q] uint8 : 1 iff the row is in collision (may be NULL)
 * Rows with a non-finite centre or a non-positive radius/semi-axis give
 * out_metric = NaN, out_collide = 0 and are reported by cs_sync.  Q == 0 is a
 * no-op.  params == NULL uses the defaults on the legacy default stream. */
CS_API cs_status cs_query(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                   float conservatism, float *out_metric, uint8_t *out_collide,
                   const cs_params *params);

/* Largest Q that cs_query_noalloc accepts. */
#define CS_QUERY_NOALLOC_MAX_ROWS 65536

/* cs_query without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc once they are
 * running -- a receding-horizon controller with a hard period, where an
 * allocation may block on the driver and synchronise the device, or a program
 * whose device memory is owned by another allocator that forbids outside
 * allocations.  Arguments, outputs and results are those of cs_query, with
 * these limits:
 *   - the scratch is one fixed area inside the library image (about 4.6 MB of
 *     device memory on every GPU that loads the library, held until the
 *     process exits), so Q <= CS_QUERY_NOALLOC_MAX_ROWS; a larger Q returns
 *     CS_ERR_INVALID_ARG before anything is enqueued;
 *   - device pointers only (params->host_io = 1 returns CS_ERR_INVALID_ARG);
 *     the scene's device must be current;
 *   - the first call on a device resolves the area's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *     The address belongs to the device's context: after cudaDeviceReset the
 *     next call resolves it again (again before any capture);
 *   - CS_METRIC_FLAGS behaves as in cs_query: out_metric, params->out_count
 *     and params->out_group_metric are not written, and with group_size > 0
 *     rows stop once their group collides (out_collide 2);
 *   - every call shares the area and it keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race and corrupt each other's rows, so the caller serialises them;
 *   - invalid rows and an expired wait show as NaN rows; cs_sync does not
 *     report them for this entry point.
 * The caller still passes the scene and every input and output buffer. */
CS_API cs_status cs_query_noalloc(const cs_scene *scene, int32_t prim_type, const float *prims,
                                  int64_t Q, float conservatism, float *out_metric,
                                  uint8_t *out_collide, const cs_params *params);

/* Adjoint of cs_query: grad_centres[j] = grad_out[j] * d metric_j / d c_j
 * ([Q,3], float).  With params->group_size > 0, grad_out has one entry per
 * group and applies to every row of the group (the group metric is a sum).
 * grad_out == NULL means ones.  The neighbour-set size is piecewise constant
 * and the Eq. 8 clamp gives zero gradient where st^2 = 0; the min mode
 * differentiates the arg-min pair.  Spheres and ellipsoids, all modes. */
CS_API cs_status cs_query_grad(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                        float conservatism, const float *grad_out, float *grad_centres,
                        const cs_params *params);

/* Forward and adjoint of cs_query in one fused launch (spheres; the mean or
 * sum cost mode): out_metric, out_collide and params->out_count,
 * out_group_metric and out_group_collide as cs_query writes them (any may be
 * NULL), and grad_centres as cs_query_grad writes it (required).  The launch
 * evaluates every pair once for both.  grad_centres has the bits of
 * cs_query_grad; the forward outputs come from the adjoint's arithmetic (the
 * square root of Eq. 8 as u rsqrt(u)), so they agree with cs_query within
 * the metric's FP32 tolerance, not bit for bit, and a pair at the edge of the
 * neighbour set or the in-collision test may be counted on the other side.
 * The adjoint's default tile shape is used whatever params->tile_config says.
 * Other primitive types or modes return CS_ERR_INVALID_ARG; a conservatism
 * sweep is rejected as for cs_query_grad.  host_io and streams as cs_query. */
CS_API cs_status cs_query_fwd_grad(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                                   float conservatism, const float *grad_out, float *out_metric,
                                   uint8_t *out_collide, float *grad_centres, const cs_params *params);

/* Pose chain for sphere robots (device pointers): for P poses (t, w) with w
 * an axis-angle rotation (Rodrigues) and K body-frame offsets p_k,
 *   out_spheres[p*K + k] = (t_p + R(w_p) p_k, radius)      [P*K, 4]  */
CS_API cs_status cs_pose_spheres(const float *poses, int64_t P, const float *offsets, int32_t K,
                          float radius, float *out_spheres, void *stream);

/* Adjoint of cs_pose_spheres: grad_poses[p] = (sum_k g_pk,
 * J_l(w_p)^T sum_k (R(w_p) p_k) x g_pk) with J_l the left Jacobian of SO(3);
 * grad_centres is [P*K,3], grad_poses [P,6] (overwritten). */
CS_API cs_status cs_pose_spheres_grad(const float *poses, int64_t P, const float *offsets, int32_t K,
                               const float *grad_centres, float *grad_poses, void *stream);

/* Wait for `stream` and report device-side conditions recorded on it since
 * the last cs_sync (CS_ERR_INVALID_ARG for invalid query rows,
 * CS_ERR_TIMEOUT for an expired wait), clearing them.  After a timeout,
 * later launches on the same stream return NaN rows without computing until
 * cs_sync clears the condition. */
CS_API cs_status cs_sync(const cs_scene *scene, void *stream);

/* Tile configurations available to cs_params.tile_config: writes up to `cap`
 * ids to `ids` and returns how many exist. */
CS_API int32_t cs_tile_configs(int32_t *ids, int32_t cap);

/* ------------------------------------------------------------------------
 * Captured query graphs.  The paper has no counterpart: this is launch
 * machinery for callers that repeat one query shape (an MPPI or optimiser
 * loop rewriting its primitives in place).
 *
 * cs_graph_create captures one cs_query call (grad_centres == NULL) or one
 * cs_query_grad call (grad_centres != NULL; out_metric and out_collide must
 * then be NULL) with the given device buffers into a CUDA graph.
 * cs_graph_launch replays it on `stream`, reading whatever the buffers hold
 * when it runs.  Arguments mean what they mean for cs_query / cs_query_grad;
 * every pointer is a device pointer (params->host_io must be 0) and
 * params->stream, params->eval_events are ignored.  The graph owns private
 * query scratch, so distinct graphs may run concurrently on different
 * streams; CUDA orders the launches of one graph.  The scene and every
 * buffer must outlive the graph.  Errors: the argument errors of cs_query,
 * CS_ERR_CUDA when capture or instantiation fails, CS_ERR_NO_MEMORY. */
typedef struct cs_graph cs_graph;

CS_API cs_status cs_graph_create(const cs_scene *scene, int32_t prim_type, const float *prims,
                                 int64_t Q, float conservatism, float *out_metric,
                                 uint8_t *out_collide, const float *grad_out, float *grad_centres,
                                 const cs_params *params, cs_graph **out);
CS_API cs_status cs_graph_launch(cs_graph *graph, void *stream);
/* Wait for `stream`, then report and clear the device-side conditions of
 * the graph's launches, as cs_sync does for a stream. */
CS_API cs_status cs_graph_sync(cs_graph *graph, void *stream);
/* Kernels one launch of the graph runs (also added to cs_launch_count by
 * every cs_graph_launch); -1 for an invalid handle. */
CS_API int64_t cs_graph_kernels(const cs_graph *graph);
/* Free the graph and its scratch; no launch of it may be in flight.  NULL
 * is a no-op. */
CS_API cs_status cs_graph_destroy(cs_graph *graph);

/* Tile autotuner.  The paper has no counterpart.  Runs the fused kernel of
 * cs_query on this batch (device pointers, as cs_query with host_io = 0)
 * with every tile configuration, one warm-up launch then `reps` (>= 1)
 * launches each timed with CUDA events on params->stream, and records the
 * fastest for (scene, prim_type, params->mode, floor(log2 Q)); calls with
 * tile_config = CS_TILE_TUNED then use it.  Writes the chosen id to *best
 * and, when ms is not NULL, the mean milliseconds per launch of the first
 * `cap` configurations in the order cs_tile_configs lists them.  Outputs of
 * the timed launches go to internal scratch.  Synchronises params->stream.
 * Errors: those of cs_query; CS_ERR_INVALID_ARG for best == NULL, reps < 1,
 * Q == 0 or host_io = 1. */
CS_API cs_status cs_autotune(cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                             float conservatism, const cs_params *params, int32_t reps,
                             int32_t *best, float *ms, int32_t cap);

/* Autotuner log.  The paper has no counterpart.  After this call every
 * cs_autotune call (any thread) appends one JSON line to the file at `path`:
 *   {"n_gaussians", "prim_type", "mode", "exact_variance", "rows" (Q),
 *    "sweep" (n_sigma blocks), "launch_rows", "reps",
 *    "ms": {"<tile id>": mean ms per launch, ...}, "best": <tile id>}
 * The file is opened, appended and closed per line; a file that cannot be
 * opened is skipped silently.  path == NULL or "" stops logging.  The path
 * is copied.  Always returns CS_OK. */
CS_API cs_status cs_autotune_log(const char *path);

/* ------------------------------------------------------------------------
 * One MPPI iteration (Section II-D) for a robot that is one sphere under
 * single-integrator (velocity) control, fused on the device: rollouts of K
 * sampled control sequences over T steps, the conservative metric of every
 * rollout position (Eq. 8, Eq. 11 averaged over the neighbour set, summed
 * over the horizon), the per-rollout cost (the sum of collision, task and
 * control terms; the paper's image term is not modelled), the Eq. 10 softmin
 * weights with temperature lambda, and the update of the nominal sequence:
 *   u[k,t] = U[t] + eps[k,t],  x[k,t+1] = x[k,t] + dt u[k,t],  x[k,0] = x0,
 *   C^k = w_collision sum_t mc(x[k,t+1]) + w_goal sum_t |x[k,t+1] - goal|^2
 *         + w_terminal |x[k,T] - goal|^2 + w_control sum_t |u[k,t]|^2,
 *   w^k = exp(-C^k / lambda) / sum_l exp(-C^l / lambda),
 *   U_out[t] = U[t] + sum_k w^k eps[k,t].
 * The perturbations eps are drawn by the caller. */
typedef struct cs_mppi_desc {
    int32_t K;            /* rollouts, 1 .. 2^20 */
    int32_t T;            /* horizon steps, 1 .. 1024 (K * T <= 2^26) */
    float dt;             /* step, > 0 */
    float radius;         /* robot sphere radius, > 0 */
    float nsigma;         /* conservatism n_sigma, >= 0 */
    float lambda;         /* Eq. 10 temperature, > 0 */
    float w_collision, w_goal, w_terminal, w_control;  /* cost weights, >= 0 */
    float goal[3];
} cs_mppi_desc;

/* Device pointers: x0 [3], U [T,3], eps [K,T,3] (row-major), U_out [T,3] (may
 * equal U), and optionally cost [K], weights [K] and collide [K] (a rollout
 * collides if any of its positions does, as cs_query's flag).  params gives
 * the metric parameters, the stream and the tile shape (NULL = defaults);
 * its mode, group and output members are ignored (the collision term is the
 * mean cost) and host_io must be 0.  Asynchronous on the stream; scratch is
 * the stream's pooled query scratch (grown once).  Non-finite inputs give
 * NaN costs.  Errors: CS_ERR_INVALID_ARG for bad sizes, weights or NULL
 * buffers, and those of cs_query. */
CS_API cs_status cs_mppi_step(const cs_scene *scene, const cs_mppi_desc *desc, const float *x0, const float *U,
                              const float *eps, float *U_out, float *cost, float *weights, uint8_t *collide,
                              const cs_params *params);

/* The same iteration captured into a query graph (see cs_graph_create):
 * every cs_graph_launch runs it again on the buffers given here, reading the
 * x0, U and eps they hold at that time (an MPPI loop writes the next
 * perturbations into eps and copies U_out to U, or passes U_out == U).
 * Launch, sync and free it with cs_graph_launch / cs_graph_sync /
 * cs_graph_destroy.  Errors: those of cs_mppi_step and cs_graph_create. */
CS_API cs_status cs_mppi_graph_create(const cs_scene *scene, const cs_mppi_desc *desc, const float *x0,
                                      const float *U, const float *eps, float *U_out, float *cost, float *weights,
                                      uint8_t *collide, const cs_params *params, cs_graph **out);

/* ------------------------------------------------------------------------
 * One batched RRT extension (Section II-E) for a robot that is one sphere of
 * radius `radius`, the tree resident in caller device buffers.  The paper
 * grows its tree 32 nodes at a time and checks every candidate edge with the
 * metric; here, for the B samples of one call:
 *   1. nearest: the closest of nodes[0, *count) to each sample (squared
 *      distance in FP32, the lowest index on ties);
 *   2. steer: the new node is the sample when it lies within `step`, else
 *      the point `step` away from the nearest node towards it;
 *   3. edge: M points from the nearest node to the new node,
 *      p_m = x_near + (new - x_near) (m + 1) / M, the last one the new node;
 *   4. check: the edge collides when one of its points does (more than
 *      params->k_thr Gaussians with st^2 < 1), evaluated in CS_METRIC_FLAGS
 *      mode, so an edge stops at its first colliding point;
 *   5. insert: the new nodes of the free edges are appended in sample order
 *      at nodes[*count ..] with parent = their nearest node, while
 *      `capacity` lasts, and *count advances.
 * Steps 1-3 use correctly rounded FP32 operations in that order (no fused
 * multiply-add), so they are exactly reproducible. */
typedef struct cs_rrt_desc {
    int32_t B;          /* samples per extension, 1 .. 1024 */
    int32_t M;          /* checked points per edge, 2 .. 1024 (B * M <= 2^20) */
    float step;         /* longest edge, > 0 */
    float radius;       /* robot sphere radius, > 0 */
    float nsigma;       /* conservatism n_sigma, >= 0 */
    int32_t capacity;   /* node capacity of nodes / parent, >= 1 */
} cs_rrt_desc;

/* Device pointers: nodes [capacity,3] and parent [capacity] (the tree, in
 * and out), count [1] (in and out; the tree needs its root, *count >= 1),
 * samples [B,3], and optionally nearest [B] (the node each sample extended)
 * and edge_free [B] (1: the edge is free and its node was offered to the
 * tree; 0: it collides).  params gives the metric parameters, k_thr, the
 * stream and the tile shape (NULL = defaults); its mode, group and output
 * members are ignored and host_io must be 0.  Asynchronous on the stream;
 * scratch is the stream's pooled query scratch.  Errors: CS_ERR_INVALID_ARG
 * for bad sizes or NULL buffers, and those of cs_query. */
CS_API cs_status cs_rrt_extend(const cs_scene *scene, const cs_rrt_desc *desc, float *nodes, int32_t *parent,
                               int32_t *count, const float *samples, int32_t *nearest, uint8_t *edge_free,
                               const cs_params *params);

/* The same extension captured into a query graph (see cs_graph_create):
 * every cs_graph_launch extends the tree held in the buffers given here with
 * the B samples `samples` holds at that time (an RRT loop writes the next
 * samples there before each launch).  The tree's node count lives in
 * `count` on the device, so consecutive launches grow it without the host.
 * Launch, sync and free it with cs_graph_launch / cs_graph_sync /
 * cs_graph_destroy.  Errors: those of cs_rrt_extend and cs_graph_create. */
CS_API cs_status cs_rrt_graph_create(const cs_scene *scene, const cs_rrt_desc *desc, float *nodes, int32_t *parent,
                                     int32_t *count, const float *samples, int32_t *nearest, uint8_t *edge_free,
                                     const cs_params *params, cs_graph **out);

/* ------------------------------------------------------------------------
 * Serving loop.  The paper has no counterpart: this is the runtime that keeps
 * scenes resident and answers collision-query requests of uneven size (one
 * RRT edge to a whole MPPI batch) for many clients.
 *
 * The server owns `slots` batch slots, each with its own CUDA stream and
 * fixed device and pinned host buffers for `slot_rows` query rows, all
 * allocated by cs_server_create (about slots x slot_rows x 140 bytes of
 * device memory and x 60 bytes of pinned host memory), so requests are
 * admitted by memory: a request waits until a slot is free, then joins that
 * slot's batch together with the other waiting requests for the same scene
 * and primitive type, in submission order, while the slot's rows and
 * max_requests allow.  A launcher thread forms a batch whenever a slot is
 * free and requests wait, so batches overlap on the device (continuous
 * batching).  Each batch is one pass of the cs_query path over the
 * concatenated rows with per-row n_sigma; a request's results are bitwise
 * those of a cs_query call on that request alone with the same parameters
 * and tile configuration. */
typedef struct cs_server cs_server;

typedef struct cs_server_config {
    int32_t slots;        /* batches in flight, 1..16 (default 3) */
    int64_t slot_rows;    /* rows one batch holds, also the largest request (default 2^19) */
    int32_t max_requests; /* requests one batch holds (default 4096) */
    int32_t tile_config;  /* as cs_params.tile_config (default CS_TILE_TUNED) */
    cs_params params;     /* metric parameters of every request: gamma, d_max, s_min, eps, tau,
                             k_thr, mode (the pointer, stream and group members are ignored) */
    int32_t use_graphs;   /* 1 (default): a batch of R rows runs the query path as a replay of
                             a CUDA graph the slot captured for (scene, primitive type, counts
                             wanted, bucket), bucket = the next power of two >= max(R, 1024)
                             capped at slot_rows, the rows past R padded with primitives far
                             outside every scene (they reach nothing and change no result);
                             0: the query path's kernels are launched one by one */
} cs_server_config;

/* One request.  Every pointer is a host pointer; `prims` is read when the
 * request is batched and the outputs are written when it completes, so all
 * of them must stay valid until cs_server_wait has returned for it. */
typedef struct cs_request {
    int32_t scene;        /* index into the scenes passed to cs_server_create */
    int32_t prim_type;    /* cs_prim_type */
    const float *prims;   /* [Q, 4] spheres or [Q, 10] ellipsoids, as for cs_query */
    int64_t Q;            /* rows, 1..slot_rows */
    float conservatism;   /* n_sigma >= 0 for every row of the request */
    int32_t group_size;   /* > 0: group outputs as cs_params.group_size */
    float *out_metric;    /* [Q] or NULL */
    uint8_t *out_collide; /* [Q] or NULL */
    int32_t *out_count;   /* [Q] or NULL */
    float *out_group_metric;    /* [ceil(Q/group_size)] or NULL */
    uint8_t *out_group_collide; /* [ceil(Q/group_size)] or NULL */
} cs_request;

/* Timeline of a completed request, in seconds of cs_server_clock. */
typedef struct cs_request_times {
    double submitted;        /* cs_server_submit accepted it */
    double launched;         /* its batch started to be assembled */
    double completed;        /* its results were in the caller's buffers */
    int64_t batch_rows;      /* rows of the batch it ran in */
    int64_t batch_requests;  /* requests of that batch */
    int32_t status;          /* cs_status of the request */
} cs_request_times;

typedef struct cs_server_stats {
    int64_t batches, rows, requests;             /* launched so far */
    int64_t max_batch_rows, max_batch_requests;
    int64_t pending;                             /* submitted, not yet batched */
    int64_t busy_slots;
} cs_server_stats;

/* Defaults as listed in cs_server_config.  CS_ERR_INVALID_ARG for NULL. */
CS_API cs_status cs_server_config_init(cs_server_config *cfg);
/* Start a server over `n_scenes` resident scenes (all on the current
 * device; they must outlive the server).  cfg NULL = defaults.  Errors:
 * CS_ERR_INVALID_ARG for bad sizes or parameters, CS_ERR_BAD_HANDLE for a
 * bad scene, CS_ERR_NO_MEMORY / CS_ERR_CUDA when the slots cannot be
 * allocated. */
CS_API cs_status cs_server_create(cs_scene *const *scenes, int32_t n_scenes, const cs_server_config *cfg,
                                  cs_server **out);
/* Queue a request and return its ticket.  The rows are validated on the host
 * first (finite values, positive radius or semi-axes): CS_ERR_INVALID_ARG
 * and nothing queued on failure.  Thread-safe. */
CS_API cs_status cs_server_submit(cs_server *server, const cs_request *req, uint64_t *ticket);
/* Wait until the request of `ticket` has completed (timeout_s < 0: no
 * limit), fill *times (may be NULL) and retire the ticket.  Returns the
 * request's status, CS_ERR_TIMEOUT when the limit ran out (the ticket stays
 * valid), CS_ERR_INVALID_ARG for an unknown ticket.  Thread-safe. */
CS_API cs_status cs_server_wait(cs_server *server, uint64_t ticket, double timeout_s, cs_request_times *times);
CS_API cs_status cs_server_stats_get(cs_server *server, cs_server_stats *out);
/* The monotonic clock of cs_request_times, in seconds. */
CS_API double cs_server_clock(void);
/* Stop the launcher, finish the batches in flight and free the server.
 * Requests not yet batched are dropped; no cs_server_wait may be in
 * progress.  NULL is a no-op. */
CS_API cs_status cs_server_destroy(cs_server *server);

/* Zeroth-order path refinement (Section III): the RRT path smoothed by one
 * MPPI step (Section II-D) whose horizon is the whole plan, over the control
 * points ("knots") of a clamped uniform cubic B-spline through it.
 *   - the curve: the control points P_0 .. P_{N-1} padded with two more
 *     copies of each endpoint (so it starts at P_0 and ends at P_{N-1}),
 *     N + 1 segments of the uniform cubic basis, each sampled at u = m / M,
 *     m < M, plus the last point: (N + 1) M + 1 spheres of `radius`;
 *   - rollout k moves the interior control points by eps[k] (the endpoints
 *     stay fixed; their perturbations are ignored);
 *   - cost C^k = w_length * (length of the polyline through the samples) +
 *     w_collision * (sum over the samples of the Eq. 11 cost averaged over
 *     the neighbour set);
 *   - Eq. 10 weights w^k and the update P' = P + sum_k w^k eps[k] (interior).
 * The sample points are computed in float32 with every operation rounded in
 * a fixed order:
 *     u = m / M, u2 = u u, u3 = u2 u, v = 1 - u;
 *     b0 = ((v v) v) / 6, b1 = ((3 u3 - 6 u2) + 4) / 6,
 *     b2 = (((3 u2 - 3 u3) + 3 u) + 1) / 6, b3 = u3 / 6;
 *     x = ((b0 Q0 + b1 Q1) + b2 Q2) + b3 Q3,
 * so they are reproducible exactly. */
typedef struct cs_refine_desc {
    int32_t K;          /* perturbed paths, [1, 2^20] */
    int32_t N;          /* control points, [2, 4096] */
    int32_t M;          /* samples per spline segment, [1, 256] */
    float radius;       /* robot sphere radius, > 0 */
    float nsigma;       /* conservatism n_sigma, >= 0 */
    float lambda;       /* Eq. 10 temperature, > 0 */
    float w_length;     /* >= 0 */
    float w_collision;  /* >= 0 */
} cs_refine_desc;

/* One refinement step on device buffers: ctrl [N,3], eps [K,N,3] (the
 * caller draws the perturbations), ctrl_out [N,3] (may not alias ctrl or
 * eps); cost and weights [K] optional (NULL: not returned).  params as for
 * cs_query (mode, group_size and the output pointers are set by the call;
 * host_io must be 0).  Scratch comes from the stream's pool. */
CS_API cs_status cs_path_refine(const cs_scene *scene, const cs_refine_desc *desc, const float *ctrl,
                                const float *eps, float *ctrl_out, float *cost, float *weights,
                                const cs_params *params);

/* ---------------------------------------------------------------------------
 * Image synthesis (Section II-A, Eq. 3-4), the terminal-state images of
 * Section II-D: the scene's kept Gaussians are projected into pinhole cameras
 * (the mean by the point projection, the covariance by Eq. 3,
 * Sigma' = J R Sigma R^T J^T with J the Jacobian of the projection at the
 * mean) and alpha-blended front to back in depth order at every pixel
 * (Eq. 4), in 16x16-pixel tiles, into device buffers (no graphics API).
 *
 * Rules the paper leaves open, fixed here:
 *   - camera: x_c = R x_w + t, looking along +z, x to the right, y down the
 *     image rows; u = fx x/z + cx, v = fy y/z + cy; pixel (i, j) samples the
 *     image point (i + 0.5, j + 0.5);
 *   - Sigma' gets `dilation` px^2 added to its diagonal (it stays invertible
 *     for 2DGS disks seen edge on); a Gaussian is drawn when its camera-frame
 *     depth is at least near_plane and det(Sigma') > 0;
 *   - G2D(x) = exp(-(x - u)^T Sigma'^-1 (x - u) / 2); a Gaussian counts at a
 *     pixel when opacity * G2D >= 1/255, that product is clamped to 0.99, and
 *     a pixel stops before the Gaussian that would bring its transmittance
 *     below 1e-4;
 *   - order: increasing float32 depth of the mean, computed as
 *     ((R[6] x + R[7] y) + R[8] z) + t[2] with each operation rounded, equal
 *     depths in the scene's internal order;
 *   - colour: one RGB per Gaussian (view independent); depth output: the
 *     blended Euclidean distance of the means from the camera centre (the
 *     colour replaced by the splat's distance); alpha output: 1 - final
 *     transmittance; the background shows through the final transmittance.
 * ------------------------------------------------------------------------- */
typedef struct cs_camera {
    float R[9];            /* world-to-camera rotation, row-major */
    float t[3];            /* x_c = R x_w + t */
    float fx, fy, cx, cy;  /* pinhole intrinsics in pixels */
} cs_camera;

typedef struct cs_render_desc {
    int32_t n_views;       /* cameras (images), >= 0 */
    int32_t width, height; /* pixels, each in [1, 4096] */
    float near_plane;      /* default 0.01 (scene units) */
    float dilation;        /* px^2 added to the diagonal of Sigma', >= 0 (default 0.3) */
    float background[3];   /* colour behind the Gaussians (default 0, 0, 0) */
    void *stream;          /* cudaStream_t */
    int64_t *out_instances;/* optional host pointer: receives the number of (view, Gaussian,
                              tile) instances the call blended from */
} cs_render_desc;

CS_API cs_status cs_render_desc_init(cs_render_desc *desc);

/* Appearance used by cs_render: per input row of cs_scene_create, its
 * opacity (NULL: 1) and RGB colour ([n,3], NULL: 1, 1, 1), gathered into the
 * scene's internal order (rows the floater filter dropped are ignored).
 * on_device: 1 device pointers, 0 host pointers.  Replaces an earlier
 * appearance; allocates the scene's appearance array on the first call and
 * returns after the stream has finished.  Values are not range-checked:
 * opacities outside [0, 1] blend as given. */
CS_API cs_status cs_scene_set_appearance(cs_scene *scene, const float *opacity, const float *colors,
                                         int32_t on_device, void *stream);

/* Render desc->n_views images (Eq. 3-4).  cams: device [n_views] cs_camera.
 * out_rgb: device [n_views, height, width, 3] (required); out_depth,
 * out_alpha: device [n_views, height, width] or NULL.  Steps: projection of
 * every (view, Gaussian) with its tile range, the (Gaussian, tile) instances
 * listed and sorted by (view, tile, depth) with a stable radix sort, then one
 * CTA per tile blending its pixels.  Scratch is pooled per (device, stream)
 * and grown on demand; the call waits for the stream once, after counting
 * the instances, to size it.  Errors: CS_ERR_INVALID_ARG for sizes out of
 * range, NULL required pointers or a scene without appearance
 * (cs_scene_set_appearance); CS_ERR_UNSUPPORTED when a call has more than
 * 2^31 instances (render fewer views per call). */
CS_API cs_status cs_render(const cs_scene *scene, const cs_render_desc *desc, const cs_camera *cams,
                           float *out_rgb, float *out_depth, float *out_alpha);

/* Self-test of the bounded-wait machinery: launches one block that waits on
 * a barrier nothing completes, with a budget of `spins` polls, and returns
 * CS_ERR_TIMEOUT when the wait gave up (the expected result) or CS_OK if it
 * did not.  Faults nothing; the context stays usable. */
CS_API cs_status cs_selftest_wait_timeout(int64_t spins, void *stream);

/* Free the pooled query scratch of every stream (grown on demand by
 * cs_query / cs_query_grad and kept for reuse; never allocated per call once
 * large enough).  No query may be in flight. */
CS_API cs_status cs_release_scratch(void);

/* Number of kernels this library has launched in this process (host-side
 * count, all threads and devices). */
CS_API int64_t cs_launch_count(void);

/* Message for the last failure on this thread ("" if none). */
CS_API const char *cs_last_error(void);

/* Library version string. */
CS_API const char *cs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CS_B300_H */
