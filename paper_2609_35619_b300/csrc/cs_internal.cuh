// cs_internal.cuh -- internal definitions shared by the CUDA sources of the
// collision-metric engine (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <unordered_map>

#include "../../include/cs_b300.h"

namespace cs {

// ---------------------------------------------------------------- constants
constexpr int kChunk = 32;             // Gaussians per chunk record (warp-level cull unit)
constexpr int kMortonBits = 8;         // bits per axis of the query sort key
constexpr int kSceneOrderBits = 10;    // bits per axis of the scene order (Hilbert index)
constexpr int kSegment = 1024;         // Gaussians per greedy chunking segment
constexpr int kSigmaBins = 512;        // log2 histogram of the largest scale
constexpr float kSigmaLog2Lo = -32.f;  // histogram covers 2^-32 .. 2^32 in 1/8 octaves
constexpr float kSigmaBinsPerOctave = 8.f;
constexpr float kReachPadRel = 1e-4f;  // relative padding of every cull radius

// A named NVTX range over the enclosing scope (host timeline): scene build,
// query preparation, the fused kernel, group epilogue, serving batches,
// autotuning.  NVTX v3 is header-only and costs a branch unless a profiler
// has attached, so the ranges are always compiled in.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// device error word bits
constexpr unsigned kErrInvalidQuery = 1u;
constexpr unsigned kErrTimeout = 2u;
constexpr unsigned kErrBounds = 4u;    // an index check of a CS_DEBUG build failed

// CS_IDX_OK(cond, err): in a CS_DEBUG build, evaluates the index condition
// `cond`; when it is false, records kErrBounds in the error word `err` and
// yields false, and the caller keeps the access in bounds: it skips it, or
// redirects it to element 0 (no trap: the context stays usable, cs_sync
// reports CS_ERR_BOUNDS, and that call's outputs are not valid).  In a
// normal build it is `true` and the condition is not evaluated.
#ifdef CS_DEBUG
#define CS_IDX_OK(cond, err) ((cond) ? true : (atomicOr((err), ::cs::kErrBounds), false))
constexpr bool kDebugBuild = true;
#else
#define CS_IDX_OK(cond, err) true
constexpr bool kDebugBuild = false;
#endif

// bounded wait: polls of mbarrier.try_wait before giving up; the waits also
// give up after one second of wall time
constexpr long long kWaitPolls = 1ll << 27;

// ------------------------------------------------------------- scene layout
// Repacked Gaussians are stored in chunk blocks of kChunk = 32 slots, one
// 1184-byte block each, so that a run of chunks is one contiguous 1-D bulk
// copy and lane l of a warp reads slot l of a chunk with conflict-free 4-byte
// shared-memory loads.  Gaussians follow a global Morton order of their means
// (10 bits per axis over the scene cube), the large tier after the rest; a
// chunk takes consecutive Gaussians while their box stays within an extent
// limit (and at most 32), so chunk boxes are compact wherever the scene is
// dense or sparse.  Unused slots are padding.
//   lo  = (min mu over the chunk, max scale over the chunk)
//   hi  = (max mu over the chunk, number of real slots)
//   x, y, z          the means
//   sxx, syy, szz    the covariance diagonal (Eq. 2)
//   sxy2, sxz2, syz2 the off-diagonals, doubled so d^T Sigma d takes 9 FP32 ops
// Padding slots hold a point at 1e18 with a zero covariance: every pair with
// it has st2 = +inf (or ~1e36) and adds exactly nothing to any reduction.
struct __align__(16) ChunkBlock {
    float4 lo;
    float4 hi;
    float x[kChunk], y[kChunk], z[kChunk];
    float sxx[kChunk], syy[kChunk], szz[kChunk];
    float sxy2[kChunk], sxz2[kChunk], syz2[kChunk];
};
static_assert(sizeof(ChunkBlock) == 1184, "chunk block layout");
static_assert(sizeof(ChunkBlock) % 16 == 0, "bulk copies move whole 16-byte units");

// Bounding record of a chunk or of a node of the chunk hierarchy: the box of
// the means below it and their largest scale (lo.w).  Node k of level 1
// covers chunks [32k, 32k + 32), node k of level 2 covers level-1 nodes
// [32k, 32k + 32), and so on: an implicit fan-out-32 tree over the Morton
// order that the query producer descends one ballot per level.
struct __align__(16) NodeBox {
    float4 lo;
    float4 hi;
};
constexpr int kLevels = 3;  // node levels above the chunks

struct SceneDev {
    const ChunkBlock *blocks = nullptr;  // [nchunks]
    const NodeBox *chead = nullptr;      // [nchunks] chunk boxes (copy of the block headers)
    const NodeBox *nodes[kLevels] = {nullptr, nullptr, nullptr};  // level 1..3
    int nnodes[kLevels] = {0, 0, 0};
    const float *smax = nullptr;         // [n_gauss] largest scale per sorted Gaussian (export only)
    const int32_t *index = nullptr;      // [n_gauss] input row per sorted Gaussian (export only)
    const int32_t *slot_of = nullptr;    // [n_gauss] slot of each sorted Gaussian (export only)
    int n_gauss = 0;      // kept Gaussians
    int nchunks = 0;      // chunks of both tiers
    int large_chunk0 = 0; // first chunk of the large tier
    float chunk_extent = 0.f;  // extent limit of a chunk of the main tier
    float sigma_tier = 0.f;    // max scale over the main tier
    float pad_abs = 0.f;       // absolute slack added to cull radii
    float bb_lo[3] = {0, 0, 0}, bb_hi[3] = {1, 1, 1};  // box used for query sort keys
};

// Per-stream scratch of the query path.  Grown on demand, never shrunk, never
// allocated per call once large enough.
struct Workspace {
    cudaStream_t stream = nullptr;
    size_t cap_q = 0;
    uint32_t *keys[2] = {nullptr, nullptr};
    uint32_t *vals[2] = {nullptr, nullptr};
    uint32_t *sort_hist = nullptr;   size_t cap_hist = 0;
    uint32_t *scan_tmp = nullptr;    size_t cap_scan_tmp = 0;
    float4 *qrec = nullptr;          // [Q * recs] prepared primitives, sorted order
    float *qns = nullptr;            // [Q] n_sigma, sorted order
    // host_io staging
    float *io_prims = nullptr;       size_t cap_io_prims = 0;
    float *io_ns = nullptr;
    float *io_metric = nullptr;
    uint8_t *io_collide = nullptr;
    int32_t *io_count = nullptr;
    float *io_grad = nullptr;
    float *io_gout = nullptr;
    float *io_gm = nullptr;
    uint8_t *io_gc = nullptr;
    // MPPI iteration scratch (cs_mppi_step): sphere centres of the rollouts
    // [K*T,4], then per rollout the collision cost and the task + control cost
    float *mppi = nullptr;           size_t cap_mppi = 0;  // floats
    // RRT extension scratch (cs_rrt_extend): edge points, nearest, new nodes, edge flags
    float *rrt = nullptr;            size_t cap_rrt = 0;   // floats
    // rendering scratch (cs_render): projections, instance lists, sort buffers
    void *rnd = nullptr;             size_t cap_rnd = 0;   // bytes: per (view, slot)
    void *rnd2 = nullptr;            size_t cap_rnd2 = 0;  // bytes: per instance
    // conservatism sweep (cs_params.sweep_count): the prepared rows before expansion
    unsigned *err = nullptr;         // device error word
};

struct Scene {
    SceneDev dev;
    // tile shapes chosen by cs_autotune, keyed by tune_key()
    std::mutex tune_mu;
    std::unordered_map<uint32_t, int32_t> tuned;
    int64_t n_input = 0, n_kept = 0, n_grid = 0, n_large = 0, n_invalid = 0;
    int64_t device_bytes = 0;
    float4 *app = nullptr;           // per slot (opacity, r, g, b) for rendering (cs_scene_set_appearance)
    void *blocks[8] = {};            // owned device allocations
    int nblocks = 0;
    int device = 0;
    int num_sms = 148;
    uint32_t magic = 0;
};

// Histogram entries the query preparation needs beyond the radix sort's
// (the small-batch counting sort over 2^16 buckets, plus its total).
constexpr size_t kPrepHistElems = (1u << 16) + 1;

// Query scratch is pooled per (device, stream) and shared by every scene
// used on that stream; it lives until cs_release_scratch or process exit.
cs_status get_workspace(int device, cudaStream_t stream, size_t Q, bool host_io, Workspace **out);
Workspace *find_workspace(int device, cudaStream_t stream);
// A workspace outside the pool (owned by a graph or a server slot).
cs_status new_workspace(cudaStream_t stream, Workspace **out);
cs_status grow_workspace(Workspace *w, size_t Q, bool host_io);
void delete_workspace(Workspace *w);

constexpr uint32_t kSceneMagic = 0xC5B300A1u;

// Key of a tuned tile shape: primitive type, metric mode and batch-size class
// floor(log2 Q).
inline uint32_t tune_key(int32_t prim_type, int32_t mode, int64_t Q) {
    uint32_t c = 0;
    while (c < 40 && (int64_t(1) << (c + 1)) <= Q) ++c;
    return (uint32_t)prim_type | ((uint32_t)mode << 2) | (c << 8);
}

// The query path behind cs_query / cs_query_grad (also captured by
// cs_graph_create and driven by the serving loop).
cs_status query_common(const cs_scene *s, int32_t prim_type, const float *prims, int64_t Q,
                       float conservatism, const cs_params *params, bool grad, float *out_metric,
                       uint8_t *out_collide, const float *grad_out, float *grad_centres,
                       Workspace *own_ws, bool fused = false);
int tile_configs(int32_t *ids, int32_t cap);
int64_t launch_total();

// One MPPI iteration (cs_mppi_step); own_ws = scratch owned by a graph.
cs_status mppi_common(const cs_scene *scene, const cs_mppi_desc *d, const float *x0, const float *U,
                      const float *eps, float *U_out, float *cost, float *weights, uint8_t *collide,
                      const cs_params *params, Workspace *own_ws);
cs_status mppi_reserve(Workspace *w, int64_t K, int64_t T);
cs_status mppi_check(const cs_scene *scene, const cs_mppi_desc *d, const float *x0, const float *U,
                     const float *eps, const float *U_out);

// One batched RRT extension (cs_rrt_extend); own_ws = scratch owned by a graph.
cs_status rrt_common(const cs_scene *scene, const cs_rrt_desc *d, float *nodes, int32_t *parent, int32_t *count,
                     const float *samples, int32_t *nearest, uint8_t *edge_free, const cs_params *params,
                     Workspace *own_ws);
cs_status rrt_reserve(Workspace *w, int B, int M);
cs_status rrt_check(const cs_scene *scene, const cs_rrt_desc *d, const float *nodes, const int32_t *parent,
                    const int32_t *count, const float *samples);

// ------------------------------------------------------- launch accounting
// Host-side count of kernel launches (cs_launch_count); every launcher adds
// the number of kernels it enqueues.
void count_launches(int n);

// ---------------------------------------------------- error helpers (host)
void set_error(const std::string &msg);
cs_status cuda_fail(cudaError_t e, const char *what);
cs_status invalid(const char *msg);
cs_status check_scene(const cs_scene *s);
cs_status check_params(const cs_params &p);
// The number of n_sigma blocks of a call (1 without a sweep).
inline int sweep_blocks(const cs_params &p) { return p.sweep_count >= 2 ? p.sweep_count : 1; }
struct SweepNs {
    float v[8];
};
// The library's stream-ordered memory pool of the current device, for
// temporaries that live within one call (the scene build): allocations and
// frees are enqueued on the caller's stream and never synchronise the
// device; up to 1 GB stays reserved between calls (cs_release_scratch trims).
cudaError_t temp_pool(cudaMemPool_t *out);
// Scratch of a sweep over Q rows: per-row outputs of S Q rows (group-only
// requests); the Q rows themselves are prepared once and copied in the kernel.
cs_status sweep_reserve(Workspace *w, int64_t Q, int prim_type, int S);

#define CS_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::cs::cuda_fail(e_, #call);      \
    } while (0)

// ---------------------------------------------------- primitives (host API)
size_t scan_tmp_elems(size_t n);
// exclusive scan of n uint32 values (in may equal out); tmp from scan_tmp_elems
void scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s);

size_t sort_hist_elems(size_t n);
// stable LSD radix sort of (keys, vals) on the low `bits` bits; the result is
// in keys[res], vals[res] where res (0 or 1) is returned.
int radix_sort(uint32_t *keys[2], uint32_t *vals[2], size_t n, int bits, uint32_t *hist,
               uint32_t *scan_tmp, cudaStream_t s);

// ------------------------------------------------------ device-side helpers
__device__ __forceinline__ int float_to_ordered(float f) {
    int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ordered_to_float(int i) {
    return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF);
}

// Group outputs (Section II-D/E): sum of the metric and OR of the flag over
// the rows [b, e) of one group.  Groups of 32 rows or more are reduced by a
// warp: lane l sums rows b + l, b + l + 32, ... in order, then a fixed xor
// tree; shorter groups by one thread in row order.  The order depends only on
// the group size, so a group's bits do not depend on the launch it is in.
constexpr int kGroupWarpMin = 32;
__device__ __forceinline__ void group_rows_warp(const float *__restrict__ metric,
                                                const uint8_t *__restrict__ collide, int b, int e,
                                                int lane, float &s, unsigned &c) {
    s = 0.f;
    c = 0u;
    for (int j = b + lane; j < e; j += 32) {
        if (metric) s += metric[j];
        if (collide) c |= collide[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        c |= __shfl_xor_sync(0xffffffffu, c, o);
    }
    c = c != 0u;  // a group collides if a row does (rows may hold 2: unfinished, group colliding)
}
__device__ __forceinline__ void group_rows_serial(const float *__restrict__ metric,
                                                  const uint8_t *__restrict__ collide, int b, int e,
                                                  float &s, unsigned &c) {
    s = 0.f;
    c = 0u;
    for (int j = b; j < e; ++j) {
        if (metric) s += metric[j];
        if (collide) c |= collide[j];
    }
    c = c != 0u;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// One poll; true when the phase with the given parity has completed.
// try_wait with a suspend-time hint: the thread may sleep up to `ns`
// nanoseconds for the phase (it resumes when the phase completes), so a long
// wait takes few polls and leaves the issue slots to other warps.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, unsigned parity, unsigned ns) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared, completing `bytes` on the mbarrier.  Both
// addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32x2 arithmetic (sm_100 family): two independent IEEE
// round-to-nearest operations per instruction, so a packed evaluation gives
// exactly the bits of two scalar ones.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Reach of a cull: every pair whose centre distance exceeds
// R(sigma) = alpha sigma + sqrt(alpha^2 sigma^2 + beta) has st^2 > S_reach,
// where (alpha, beta) come from the primitive (see prepare kernels).
// EX (exact variance of the quadratic form): the trace term adds at most
// 1.5 sigma^4 (scaled like the rest) under the root of sigma^2, and the
// condition x^2 - 2 alpha sqrt(sigma^2 x^2 + 1.5 sigma^4) <= beta on the
// centre distance x solves to
//   x^2 <= beta + 2 a^2 + 2 a sqrt(beta + a^2 + 1.5 sigma^2),  a = alpha sigma,
// which reduces to R(sigma)^2 without the 1.5 sigma^2.  Both grow with alpha
// and beta, so the largest of a group bound the whole group.
// The roots are the hardware approximation (one MUFU operation, relative
// error below 2^-22); the relative padding kReachPadRel = 1e-4 covers it
// many times over, so the radius stays an upper bound.  Its input is held at
// FLT_MIN or above (the approximation flushes subnormals to zero, which would
// make a tiny radius smaller than it is).
template <bool EX = false>
__device__ __forceinline__ float reach(float alpha, float beta, float sigma, float pad_abs) {
    float a = alpha * sigma;
    if constexpr (EX) {
        const float inner = sqrt_approx(fmaxf(fmaf(a, a, fmaf(1.5f * sigma, sigma, beta)), FLT_MIN));
        return sqrt_approx(fmaxf(fmaf(2.f * a, a + inner, beta), FLT_MIN)) * (1.f + kReachPadRel) + pad_abs;
    }
    return (a + sqrt_approx(fmaxf(fmaf(a, a, beta), FLT_MIN))) * (1.f + kReachPadRel) + pad_abs;
}

}  // namespace cs
