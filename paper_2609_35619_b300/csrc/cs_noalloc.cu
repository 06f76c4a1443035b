// cs_noalloc.cu -- cs_query_noalloc: the query path of cs_query run on one
// fixed scratch area that is part of the library image, so that a call never
// allocates device memory.
//
// Who needs it: callers that must not call cudaMalloc once they are running,
// for example a receding-horizon controller with a hard period (an allocation
// can block on the driver and synchronise the device, missing the deadline),
// or a host program whose device memory is owned by another allocator or pool
// that forbids allocations from outside it.
//
// The scratch is a file-scope static device array (kNoAllocBytes, about
// 4.6 MB); every GPU that loads the library holds it until the process exits.
// Host code only ever sees a host-side stand-in for its name, so the device
// address is resolved once per device with cudaGetSymbolAddress (on the first
// call on that device, which therefore has to come before any stream capture)
// and passed to the kernels.  The address belongs to the device's current
// context: after cudaDeviceReset (or under another context on the same
// device) the next call resolves it again.  All calls share the one area and
// it keeps the last call's contents: calls whose work overlaps on the GPU race
// with each other and must be serialised by the caller.
#include <mutex>

#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

void launch_prep(const float *prims, int prim_type, int Q, const SceneDev &sc, float ns_scalar,
                 const float *ns_rows, Workspace &ws, uint32_t **perm_out, cudaStream_t s);
void launch_group(const float *metric, const uint8_t *collide, int Q, int G, float *gm, uint8_t *gc,
                  cudaStream_t s, unsigned *err = nullptr);
cudaError_t run_eval(int prim_type, const SceneDev &sc, const float4 *qrec, const float *qns,
                     const uint32_t *perm, int Q, const cs_params &p, float *out_metric,
                     uint8_t *out_collide, int32_t *out_count, const float *grad_out,
                     float *grad_centres, unsigned *err, int num_sms, long long polls,
                     cudaStream_t s, unsigned *gflags = nullptr);

namespace {

constexpr size_t kRows = CS_QUERY_NOALLOC_MAX_ROWS;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
// parts of the area: sort keys and rows (double-buffered), radix histograms,
// scan partials, prepared rows (up to three float4 per row), n_sigma per row,
// per-row metric and flag for group-only requests, the error word
constexpr size_t kKeyBytes = align256(4 * kRows);
constexpr size_t kHistElems = 256 * (kRows / 4096 + 1) > kPrepHistElems ? 256 * (kRows / 4096 + 1)
                                                                          : kPrepHistElems;
constexpr size_t kHistBytes = align256(4 * kHistElems);
constexpr size_t kScanElems = 1024;
constexpr size_t kScanBytes = align256(4 * kScanElems);
constexpr size_t kRecBytes = align256(48 * kRows);
constexpr size_t kNsBytes = align256(4 * kRows);
constexpr size_t kMetricBytes = align256(4 * kRows);
constexpr size_t kFlagBytes = align256(kRows);
constexpr size_t kErrBytes = 256;
constexpr size_t kNoAllocBytes = 4 * kKeyBytes + kHistBytes + kScanBytes + kRecBytes + kNsBytes +
                                 kMetricBytes + kFlagBytes + kErrBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_base[kMaxDevices] = {};
void *g_ctx[kMaxDevices] = {};  // the context g_base[d] was resolved in

// The current driver context (an opaque handle; nullptr when the driver call
// is unavailable, and then the first address per device is kept).
void *current_context() {
    using Fn = int (*)(void **);
    static Fn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<Fn>(f);
    }();
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of the scratch on `device` (which must be current): resolved
// once per device and context.
cs_status scratch_base(int device, unsigned char **out) {
    if (device < 0 || device >= kMaxDevices) return invalid("device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    void *ctx = current_context();
    if (!g_base[device] || (ctx && ctx != g_ctx[device])) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
        g_base[device] = static_cast<unsigned char *>(p);
        g_ctx[device] = current_context();  // the lookup may have created the primary context
    }
    *out = g_base[device];
    return CS_OK;
}

}  // namespace
}  // namespace cs

using namespace cs;

extern "C" cs_status cs_query_noalloc(const cs_scene *scene, int32_t prim_type, const float *prims,
                                      int64_t Q, float conservatism, float *out_metric,
                                      uint8_t *out_collide, const cs_params *params) {
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if ((st = check_params(p)) != CS_OK) return st;
    if (p.host_io) return invalid("cs_query_noalloc takes device pointers only (host_io must be 0)");
    if (p.sweep_count >= 2) return invalid("cs_query_noalloc takes no conservatism sweep");
    if (prim_type != CS_PRIM_SPHERE && prim_type != CS_PRIM_ELLIPSOID)
        return invalid("prim_type must be CS_PRIM_SPHERE or CS_PRIM_ELLIPSOID");
    if (Q < 0 || Q > (int64_t)kRows)
        return invalid("Q out of range: cs_query_noalloc takes at most CS_QUERY_NOALLOC_MAX_ROWS (65536) rows");
    if (!p.nsigma_per_query && (!(conservatism >= 0.f) || !isfinite(conservatism)))
        return invalid("conservatism (n_sigma) must be finite and >= 0");
    const bool flags = p.mode == CS_METRIC_FLAGS;
    if (flags) {  // only collision flags are computed, as in cs_query
        out_metric = nullptr;
        p.out_count = nullptr;
        p.out_group_metric = nullptr;
    }
    if (Q == 0) return CS_OK;
    if (!prims) return invalid("prims is NULL");
    const bool has_group = p.group_size > 0 && (p.out_group_metric || p.out_group_collide);
    if (!out_metric && !has_group && !out_collide && !p.out_count) return invalid("no output requested");
    int dev = -1;
    CS_CUDA(cudaGetDevice(&dev));
    if (dev != sc->device) return invalid("the scene's device must be the current device");
    unsigned char *base = nullptr;
    if ((st = scratch_base(dev, &base)) != CS_OK) return st;
    if (std::max(sort_hist_elems((size_t)Q), kPrepHistElems) > kHistElems ||
        scan_tmp_elems(kHistElems) > kScanElems)
        return invalid("internal: no-allocation scratch layout too small");

    // carve the area (no allocation): the same buffers cs_query takes from its pool
    Workspace w;
    unsigned char *c = base;
    w.keys[0] = reinterpret_cast<uint32_t *>(c); c += kKeyBytes;
    w.keys[1] = reinterpret_cast<uint32_t *>(c); c += kKeyBytes;
    w.vals[0] = reinterpret_cast<uint32_t *>(c); c += kKeyBytes;
    w.vals[1] = reinterpret_cast<uint32_t *>(c); c += kKeyBytes;
    w.sort_hist = reinterpret_cast<uint32_t *>(c); c += kHistBytes;
    w.scan_tmp = reinterpret_cast<uint32_t *>(c); c += kScanBytes;
    w.qrec = reinterpret_cast<float4 *>(c); c += kRecBytes;
    w.qns = reinterpret_cast<float *>(c); c += kNsBytes;
    w.io_metric = reinterpret_cast<float *>(c); c += kMetricBytes;
    w.io_collide = reinterpret_cast<uint8_t *>(c); c += kFlagBytes;
    w.err = reinterpret_cast<unsigned *>(c);
    w.cap_q = kRows;

    cudaStream_t stream = (cudaStream_t)p.stream;
    // the area keeps the previous call's contents; the error word must start at zero
    // (every other part is fully written before it is read)
    CS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(unsigned), stream));
    float *d_metric = out_metric;
    uint8_t *d_col = out_collide;
    if (has_group) {
        if (p.out_group_metric && !d_metric) d_metric = w.io_metric;
        if (p.out_group_collide && !d_col) d_col = w.io_collide;
    }
    // flags mode with groups: one word per group, set once a row of it
    // collides (the other rows then stop); it must start at zero.  The
    // per-row metric part of the area is free in this mode.
    unsigned *gflags = nullptr;
    if (flags && p.group_size > 0) {
        gflags = reinterpret_cast<unsigned *>(w.io_metric);
        const size_t ng = (size_t)((Q + p.group_size - 1) / p.group_size);
        CS_CUDA(cudaMemsetAsync(gflags, 0, 4 * ng, stream));
    }
    uint32_t *perm = nullptr;
    launch_prep(prims, prim_type, (int)Q, sc->dev, conservatism, p.nsigma_per_query, w, &perm, stream);
    CS_CUDA(cudaGetLastError());
    CS_CUDA(run_eval(prim_type, sc->dev, w.qrec, w.qns, perm, (int)Q, p, d_metric, d_col, p.out_count,
                     nullptr, nullptr, w.err, sc->num_sms, kWaitPolls, stream, gflags));
    if (has_group) {
        launch_group(d_metric, d_col, (int)Q, p.group_size, p.out_group_metric, p.out_group_collide, stream);
        CS_CUDA(cudaGetLastError());
    }
    return CS_OK;
}
