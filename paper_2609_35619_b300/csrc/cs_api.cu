// cs_api.cu -- the C ABI declared in include/cs_b300.h: argument checking,
// scene lifetime, per-stream scratch, host<->device staging and launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>

#include "cs_internal.cuh"

namespace cs {

// implemented in the other translation units
cs_status build_scene(const cs_scene_desc *d, cudaStream_t s, Scene *sc);
void launch_prep(const float *prims, int prim_type, int Q, const SceneDev &sc, float ns_scalar,
                 const float *ns_rows, Workspace &ws, uint32_t **perm_out, cudaStream_t s);
void launch_group(const float *metric, const uint8_t *collide, int Q, int G, float *gm, uint8_t *gc,
                  cudaStream_t s, unsigned *err = nullptr);
int tile_configs(int32_t *ids, int32_t cap);
void launch_pose(const float *poses, int64_t P, const float *offsets, int K, float radius,
                 float *out, cudaStream_t s);
void launch_pose_grad(const float *poses, int64_t P, const float *offsets, int K, const float *gc,
                      float *gp, cudaStream_t s);
cudaError_t run_eval(int prim_type, const SceneDev &sc, const float4 *qrec, const float *qns,
                     const uint32_t *perm, int Q, const cs_params &p, float *out_metric,
                     uint8_t *out_collide, int32_t *out_count, const float *grad_out,
                     float *grad_centres, unsigned *err, int num_sms, long long polls,
                     cudaStream_t s, unsigned *gflags = nullptr);
cudaError_t run_wait_selftest(long long polls, unsigned *err, cudaStream_t s);
void launch_export(const SceneDev &sc, float *pos, float *cov, int32_t *index, cudaStream_t s);

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_err = msg; }

cs_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? CS_ERR_NO_MEMORY : CS_ERR_CUDA;
}

cs_status invalid(const char *msg) {
    g_err = msg;
    return CS_ERR_INVALID_ARG;
}

constexpr int64_t kMaxRows = (int64_t)1 << 30;

static void free_ws(Workspace *w) {
    void *ptrs[] = {w->keys[0], w->keys[1], w->vals[0], w->vals[1], w->sort_hist, w->scan_tmp,
                    w->qrec, w->qns, w->io_prims, w->io_ns, w->io_metric, w->io_collide,
                    w->io_count, w->io_grad, w->io_gout, w->io_gm, w->io_gc, w->mppi, w->rrt, w->rnd, w->rnd2, w->err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete w;
}

// Scratch for Q rows on `stream`, grown (never shrunk) as needed: sort keys,
// prepared primitives, per-row metric/flag buffers for group-only requests,
// and (host_io) staging for every input and output.
struct WsKey {
    int dev;
    cudaStream_t s;
    bool operator==(const WsKey &o) const { return dev == o.dev && s == o.s; }
};
struct WsHash {
    size_t operator()(const WsKey &k) const {
        return std::hash<void *>()((void *)k.s) ^ (std::hash<int>()(k.dev) << 1);
    }
};
static std::mutex g_ws_mu;
static std::unordered_map<WsKey, Workspace *, WsHash> g_ws;

Workspace *find_workspace(int device, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto it = g_ws.find(WsKey{device, stream});
    return it == g_ws.end() ? nullptr : it->second;
}

static std::mutex g_pool_mu;
static std::unordered_map<int, cudaMemPool_t> g_pools;

cudaError_t temp_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = 1ull << 30;
        if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        it = g_pools.emplace(dev, pool).first;
    }
    *out = it->second;
    return cudaSuccess;
}

static void trim_temp_pools() {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto &kv : g_pools) cudaMemPoolTrimTo(kv.second, 0);
}

cs_status new_workspace(cudaStream_t stream, Workspace **out) {
    Workspace *w = new Workspace();
    w->stream = stream;
    // the error word, then the tile counter of persistent kernel shapes
    cudaError_t e = cudaMalloc(&w->err, 2 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(w->err, 0, 2 * sizeof(unsigned), stream);
    if (e != cudaSuccess) {
        free_ws(w);
        return cuda_fail(e, "workspace error word");
    }
    *out = w;
    return CS_OK;
}

void delete_workspace(Workspace *w) {
    if (w) free_ws(w);
}

cs_status get_workspace(int device, cudaStream_t stream, size_t Q, bool host_io, Workspace **out) {
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace *&w = g_ws[WsKey{device, stream}];
    if (!w) {
        cs_status st = new_workspace(stream, &w);
        if (st != CS_OK) {
            g_ws.erase(WsKey{device, stream});
            return st;
        }
    }
    *out = w;
    return grow_workspace(w, Q, host_io);
}

cs_status sweep_reserve(Workspace *w, int64_t Q, int prim_type, int S) {
    (void)prim_type;
    return grow_workspace(w, (size_t)(Q * S), false);
}

cs_status grow_workspace(Workspace *w, size_t Q, bool host_io) {
    if (Q > w->cap_q) {
        size_t cap = std::max<size_t>({Q, 1024, w->cap_q + w->cap_q / 2});
        void *olds[] = {w->keys[0], w->keys[1], w->vals[0], w->vals[1], w->sort_hist, w->scan_tmp,
                        w->qrec, w->qns, w->io_metric, w->io_collide};
        for (void *p : olds)
            if (p) CS_CUDA(cudaFree(p));
        CS_CUDA(cudaMalloc(&w->keys[0], 4 * cap));
        CS_CUDA(cudaMalloc(&w->keys[1], 4 * cap));
        CS_CUDA(cudaMalloc(&w->vals[0], 4 * cap));
        CS_CUDA(cudaMalloc(&w->vals[1], 4 * cap));
        w->cap_hist = std::max(sort_hist_elems(cap), kPrepHistElems);
        CS_CUDA(cudaMalloc(&w->sort_hist, 4 * w->cap_hist));
        w->cap_scan_tmp = scan_tmp_elems(w->cap_hist);
        CS_CUDA(cudaMalloc(&w->scan_tmp, 4 * w->cap_scan_tmp));
        CS_CUDA(cudaMalloc(&w->qrec, 48 * cap));
        CS_CUDA(cudaMalloc(&w->qns, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_metric, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_collide, cap));
        w->cap_q = cap;
    }
    if (host_io && Q > w->cap_io_prims) {
        size_t cap = std::max(w->cap_q, Q);
        void *olds[] = {w->io_prims, w->io_ns, w->io_count, w->io_grad, w->io_gout, w->io_gm, w->io_gc};
        for (void *p : olds)
            if (p) CS_CUDA(cudaFree(p));
        CS_CUDA(cudaMalloc(&w->io_prims, 40 * cap));
        CS_CUDA(cudaMalloc(&w->io_ns, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_count, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_grad, 12 * cap));
        CS_CUDA(cudaMalloc(&w->io_gout, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_gm, 4 * cap));
        CS_CUDA(cudaMalloc(&w->io_gc, cap));
        w->cap_io_prims = cap;
    }
    return CS_OK;
}

cs_status check_scene(const cs_scene *s) {
    const Scene *sc = reinterpret_cast<const Scene *>(s);
    if (!sc || sc->magic != kSceneMagic) {
        g_err = "invalid scene handle";
        return CS_ERR_BAD_HANDLE;
    }
    return CS_OK;
}

cs_status check_params(const cs_params &p) {
    if (!(p.gamma > 0.f) || !isfinite(p.gamma)) return invalid("gamma must be finite and > 0");
    if (!isfinite(p.d_max)) return invalid("d_max must be finite");
    if (!isfinite(p.s_min)) return invalid("s_min must be finite");
    if (!(p.eps > 0.f && p.eps < 1.f)) return invalid("eps must lie in (0, 1)");
    if (!(p.tau > 0.f) || !isfinite(p.tau)) return invalid("tau must be finite and > 0");
    if (p.k_thr < 0) return invalid("k_thr must be >= 0");
    if (p.mode < 0 || p.mode > 4) return invalid("mode must be a cs_metric_mode");
    if (p.group_size < 0) return invalid("group_size must be >= 0");
    if (p.host_io != 0 && p.host_io != 1) return invalid("host_io must be 0 or 1");
    if (p.exact_variance != 0 && p.exact_variance != 1) return invalid("exact_variance must be 0 or 1");
    if (p.sweep_count < 0 || p.sweep_count > 8) return invalid("sweep_count must lie in [0, 8]");
    for (int k = 0; k < p.sweep_count && p.sweep_count >= 2; ++k)
        if (!(p.sweep_nsigma[k] >= 0.f) || !isfinite(p.sweep_nsigma[k]))
            return invalid("sweep_nsigma values must be finite and >= 0");
    if (p.tile_config != 0 && p.tile_config != CS_TILE_TUNED) {
        int32_t ids[64];
        int n = tile_configs(ids, 64);
        bool found = false;
        for (int i = 0; i < n; ++i) found |= ids[i] == p.tile_config;
        if (!found) return invalid("unknown tile_config");
    }
    return CS_OK;
}


}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_params_init(cs_params *p) {
    if (!p) return invalid("params is NULL");
    memset(p, 0, sizeof(*p));
    p->gamma = 5.f;
    p->d_max = 1.f;
    p->s_min = 1.f;
    p->eps = 1e-6f;
    p->tau = 0.05f;
    p->k_thr = 0;
    p->mode = CS_METRIC_MEAN_COST;
    return CS_OK;
}

cs_status cs_scene_create(const cs_scene_desc *desc, void *stream, cs_scene **out) {
    NvtxRange range("cs.scene_create");
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    if (!desc) return invalid("desc is NULL");
    if (desc->n < 0 || desc->n > kMaxRows) return invalid("n out of range [0, 2^30]");
    if (desc->n > 0 && (!desc->means || !desc->scales || !desc->quats))
        return invalid("means, scales and quats are required when n > 0");
    if (desc->on_device != 0 && desc->on_device != 1) return invalid("on_device must be 0 or 1");
    if (desc->use_filter && (!isfinite(desc->opacity_min) || !isfinite(desc->extent_max)))
        return invalid("floater-filter thresholds must be finite");
    if (!(desc->cell_size >= 0.f) || !isfinite(desc->cell_size)) return invalid("cell_size must be >= 0");
    if (!(desc->tier_quantile >= 0.f && desc->tier_quantile <= 1.f))
        return invalid("tier_quantile must lie in [0, 1]");
    Scene *sc = new Scene();
    CS_CUDA(cudaGetDevice(&sc->device));
    CS_CUDA(cudaDeviceGetAttribute(&sc->num_sms, cudaDevAttrMultiProcessorCount, sc->device));
    cs_status st = build_scene(desc, (cudaStream_t)stream, sc);
    if (st != CS_OK) {
        for (int i = 0; i < sc->nblocks; ++i) cudaFree(sc->blocks[i]);
        delete sc;
        return st;
    }
    sc->magic = kSceneMagic;
    *out = reinterpret_cast<cs_scene *>(sc);
    return CS_OK;
}

cs_status cs_scene_destroy(cs_scene *s) {
    if (!s) return CS_OK;
    cs_status st = check_scene(s);
    if (st != CS_OK) return st;
    Scene *sc = reinterpret_cast<Scene *>(s);
    sc->magic = 0;
    for (int i = 0; i < sc->nblocks; ++i) cudaFree(sc->blocks[i]);
    if (sc->app) cudaFree(sc->app);
    delete sc;
    return CS_OK;
}

cs_status cs_scene_info_get(const cs_scene *s, cs_scene_info *info) {
    cs_status st = check_scene(s);
    if (st != CS_OK) return st;
    if (!info) return invalid("info is NULL");
    const Scene *sc = reinterpret_cast<const Scene *>(s);
    info->n_input = sc->n_input;
    info->n_kept = sc->n_kept;
    info->n_grid = sc->n_grid;
    info->n_large = sc->n_large;
    info->n_invalid = sc->n_invalid;
    for (int k = 0; k < 3; ++k) {
        info->dims[k] = sc->dev.nnodes[k];
        info->lo[k] = sc->dev.bb_lo[k];
        info->hi[k] = sc->dev.bb_hi[k];
    }
    info->cell_size = sc->dev.chunk_extent;
    info->sigma_tier = sc->dev.sigma_tier;
    info->device_bytes = sc->device_bytes;
    return CS_OK;
}

cs_status cs_scene_export(const cs_scene *s, float *pos, float *cov, int32_t *index, void *stream) {
    cs_status st = check_scene(s);
    if (st != CS_OK) return st;
    const Scene *sc = reinterpret_cast<const Scene *>(s);
    cudaStream_t cs_ = (cudaStream_t)stream;
    const int64_t n = sc->n_kept;
    if (n == 0) return CS_OK;
    launch_export(sc->dev, pos, cov, index, cs_);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // extern "C"

namespace cs {
cs_status query_common(const cs_scene *s, int32_t prim_type, const float *prims, int64_t Q,
                       float conservatism, const cs_params *params, bool grad, float *out_metric,
                       uint8_t *out_collide, const float *grad_out, float *grad_centres,
                       Workspace *own_ws, bool fused) {
    cs_status st = check_scene(s);
    if (st != CS_OK) return st;
    Scene *sc = reinterpret_cast<Scene *>(const_cast<cs_scene *>(s));
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if ((st = check_params(p)) != CS_OK) return st;
    if (prim_type != CS_PRIM_SPHERE && prim_type != CS_PRIM_ELLIPSOID)
        return invalid("prim_type must be CS_PRIM_SPHERE or CS_PRIM_ELLIPSOID");
    if (Q < 0 || Q > kMaxRows) return invalid("Q out of range [0, 2^30]");
    if (p.tile_config == CS_TILE_TUNED) {
        std::lock_guard<std::mutex> lk(sc->tune_mu);
        auto it = sc->tuned.find(tune_key(prim_type, p.mode, Q * sweep_blocks(p)));  // the launch's rows
        p.tile_config = it == sc->tuned.end() ? 0 : it->second;
    }
    const int S = sweep_blocks(p);
    if (S > 1) {
        if (grad) return invalid("a conservatism sweep has no gradient");
        if (p.mode == CS_METRIC_FLAGS) return invalid("the flags mode takes no conservatism sweep");
        if (p.host_io) return invalid("a conservatism sweep takes device buffers (host_io must be 0)");
        if (p.nsigma_per_query) return invalid("a conservatism sweep takes no nsigma_per_query");
        if (Q * S > kMaxRows) return invalid("Q * sweep_count out of range [0, 2^30]");
    } else if (!p.nsigma_per_query && (!(conservatism >= 0.f) || !isfinite(conservatism))) {
        return invalid("conservatism (n_sigma) must be finite and >= 0");
    }
    const bool flags = p.mode == CS_METRIC_FLAGS;
    if (flags && grad) return invalid("the flags mode has no gradient");
    if (fused && prim_type != CS_PRIM_SPHERE) return invalid("the fused forward and adjoint takes spheres");
    if (fused && p.mode != CS_METRIC_MEAN_COST && p.mode != CS_METRIC_SUM_COST)
        return invalid("the fused forward and adjoint takes the mean or sum cost mode");
    if (flags) {  // only collision flags are computed
        out_metric = nullptr;
        p.out_count = nullptr;
        p.out_group_metric = nullptr;
    }
    if (Q == 0) return CS_OK;
    if (!prims) return invalid("prims is NULL");
    const bool has_group = p.group_size > 0 && (p.out_group_metric || p.out_group_collide);
    if (!grad && !out_metric && !has_group && !out_collide && !p.out_count)
        return invalid("no output requested");
    if (grad && !grad_centres) return invalid("grad_centres is NULL");
    const int stride = prim_type == CS_PRIM_SPHERE ? 4 : 10;
    cudaStream_t stream = (cudaStream_t)p.stream;

    if (p.host_io) {
        // host-side validation of the rows before anything is copied
        for (int64_t j = 0; j < Q; ++j) {
            const float *r = prims + j * stride;
            for (int a = 0; a < stride; ++a)
                if (!isfinite(r[a])) return invalid("non-finite value in prims");
            if (prim_type == CS_PRIM_SPHERE ? !(r[3] > 0.f) : !(r[7] > 0.f && r[8] > 0.f && r[9] > 0.f))
                return invalid("non-positive radius or semi-axis in prims");
            if (p.nsigma_per_query && !(p.nsigma_per_query[j] >= 0.f && isfinite(p.nsigma_per_query[j])))
                return invalid("nsigma_per_query must be finite and >= 0");
        }
    }
    Workspace *ws = own_ws;
    if (ws) {
        if ((st = grow_workspace(ws, (size_t)Q, p.host_io != 0)) != CS_OK) return st;
    } else if ((st = get_workspace(sc->device, stream, (size_t)Q, p.host_io != 0, &ws)) != CS_OK) {
        return st;
    }
    if (S > 1 && (st = sweep_reserve(ws, Q, prim_type, S)) != CS_OK) return st;

    const float *d_prims = prims, *d_ns = p.nsigma_per_query, *d_gout = grad_out;
    float *d_metric = out_metric, *d_grad = grad_centres, *d_gm = p.out_group_metric;
    uint8_t *d_col = out_collide, *d_gc = p.out_group_collide;
    int32_t *d_cnt = p.out_count;
    const int ng = p.group_size > 0 ? (int)((Q + p.group_size - 1) / p.group_size) : 0;  // per n_sigma block
    if (p.host_io) {
        CS_CUDA(cudaMemcpyAsync(ws->io_prims, prims, 4 * stride * Q, cudaMemcpyHostToDevice, stream));
        d_prims = ws->io_prims;
        if (d_ns) {
            CS_CUDA(cudaMemcpyAsync(ws->io_ns, d_ns, 4 * Q, cudaMemcpyHostToDevice, stream));
            d_ns = ws->io_ns;
        }
        if (grad && d_gout) {
            int64_t n = p.group_size > 0 ? ng : Q;
            CS_CUDA(cudaMemcpyAsync(ws->io_gout, d_gout, 4 * n, cudaMemcpyHostToDevice, stream));
            d_gout = ws->io_gout;
        }
        if (d_metric) d_metric = ws->io_metric;
        if (d_col) d_col = ws->io_collide;
        if (d_cnt) d_cnt = ws->io_count;
        if (d_grad) d_grad = ws->io_grad;
        if (d_gm) d_gm = ws->io_gm;
        if (d_gc) d_gc = ws->io_gc;
    }
    const bool fwd_out = !grad || fused;  // the launch writes forward outputs
    if (fwd_out && has_group) {
        if (d_gm && !d_metric) d_metric = ws->io_metric;
        if (d_gc && !d_col) d_col = ws->io_collide;
    }

    uint32_t *perm = nullptr;
    {
        NvtxRange r("cs.query.prep");
        launch_prep(d_prims, prim_type, (int)Q, sc->dev, S > 1 ? 0.f : conservatism, d_ns, *ws, &perm, stream);
    }
    CS_CUDA(cudaGetLastError());
    // a sweep's S copies of every sorted row are launch rows p S + s, made in
    // the kernel from the one prepared row: one tile holds all n_sigma values
    // of its primitives, which share staged chunks
    const float4 *rows = ws->qrec;
    const float *rows_ns = ws->qns;
    const int64_t Qrows = Q * S;
    unsigned *gflags = nullptr;  // flags mode: a row of the group collides (early exit of the others)
    if (flags && p.group_size > 0) {
        gflags = reinterpret_cast<unsigned *>(ws->io_metric);
        CS_CUDA(cudaMemsetAsync(gflags, 0, 4 * (size_t)ng, stream));
    }
    {
        NvtxRange r(grad ? "cs.query.eval_adjoint" : "cs.query.eval");
        CS_CUDA(run_eval(prim_type, sc->dev, rows, rows_ns, perm, (int)Qrows, p, fwd_out ? d_metric : nullptr,
                         fwd_out ? d_col : nullptr, fwd_out ? d_cnt : nullptr, d_gout, grad ? d_grad : nullptr,
                         ws->err, sc->num_sms, kWaitPolls, stream, gflags));
    }
    if (fwd_out && has_group) {
        NvtxRange r("cs.query.group");
        for (int b = 0; b < S; ++b)  // groups within each n_sigma block
            launch_group(d_metric ? d_metric + (size_t)b * Q : nullptr, d_col ? d_col + (size_t)b * Q : nullptr,
                         (int)Q, p.group_size, d_gm ? d_gm + (size_t)b * ng : nullptr,
                         d_gc ? d_gc + (size_t)b * ng : nullptr, stream, ws->err);
        CS_CUDA(cudaGetLastError());
    }
    if (p.host_io) {
        if (grad) CS_CUDA(cudaMemcpyAsync(grad_centres, d_grad, 12 * Q, cudaMemcpyDeviceToHost, stream));
        if (fwd_out) {
            if (out_metric) CS_CUDA(cudaMemcpyAsync(out_metric, d_metric, 4 * Q, cudaMemcpyDeviceToHost, stream));
            if (out_collide) CS_CUDA(cudaMemcpyAsync(out_collide, d_col, Q, cudaMemcpyDeviceToHost, stream));
            if (p.out_count) CS_CUDA(cudaMemcpyAsync(p.out_count, d_cnt, 4 * Q, cudaMemcpyDeviceToHost, stream));
            if (p.out_group_metric)
                CS_CUDA(cudaMemcpyAsync(p.out_group_metric, d_gm, 4 * ng, cudaMemcpyDeviceToHost, stream));
            if (p.out_group_collide)
                CS_CUDA(cudaMemcpyAsync(p.out_group_collide, d_gc, ng, cudaMemcpyDeviceToHost, stream));
        }
        CS_CUDA(cudaStreamSynchronize(stream));
    }
    return CS_OK;
}
}  // namespace cs

extern "C" {

cs_status cs_query(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                   float conservatism, float *out_metric, uint8_t *out_collide,
                   const cs_params *params) {
    return query_common(scene, prim_type, prims, Q, conservatism, params, false, out_metric,
                        out_collide, nullptr, nullptr, nullptr);
}

cs_status cs_query_grad(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                        float conservatism, const float *grad_out, float *grad_centres,
                        const cs_params *params) {
    return query_common(scene, prim_type, prims, Q, conservatism, params, true, nullptr, nullptr,
                        grad_out, grad_centres, nullptr);
}

cs_status cs_query_fwd_grad(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                            float conservatism, const float *grad_out, float *out_metric, uint8_t *out_collide,
                            float *grad_centres, const cs_params *params) {
    return query_common(scene, prim_type, prims, Q, conservatism, params, true, out_metric, out_collide,
                        grad_out, grad_centres, nullptr, true);
}

cs_status cs_pose_spheres(const float *poses, int64_t P, const float *offsets, int32_t K,
                          float radius, float *out_spheres, void *stream) {
    if (P < 0 || K < 0 || P * (int64_t)K > kMaxRows) return invalid("P*K out of range");
    if (!(radius > 0.f) || !isfinite(radius)) return invalid("radius must be finite and > 0");
    if (P == 0 || K == 0) return CS_OK;
    if (!poses || !offsets || !out_spheres) return invalid("NULL pointer");
    launch_pose(poses, P, offsets, K, radius, out_spheres, (cudaStream_t)stream);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

cs_status cs_pose_spheres_grad(const float *poses, int64_t P, const float *offsets, int32_t K,
                               const float *grad_centres, float *grad_poses, void *stream) {
    if (P < 0 || K < 0 || P * (int64_t)K > kMaxRows) return invalid("P*K out of range");
    if (P == 0) return CS_OK;
    if (!poses || !grad_poses || (K > 0 && (!offsets || !grad_centres))) return invalid("NULL pointer");
    launch_pose_grad(poses, P, offsets, K, grad_centres, grad_poses, (cudaStream_t)stream);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

cs_status cs_sync(const cs_scene *s, void *stream) {
    cs_status st = check_scene(s);
    if (st != CS_OK) return st;
    Scene *sc = reinterpret_cast<Scene *>(const_cast<cs_scene *>(s));
    cudaStream_t cs_ = (cudaStream_t)stream;
    CS_CUDA(cudaStreamSynchronize(cs_));
    Workspace *w = find_workspace(sc->device, cs_);
    if (!w) return CS_OK;
    unsigned e = 0;
    CS_CUDA(cudaMemcpyAsync(&e, w->err, sizeof(e), cudaMemcpyDeviceToHost, cs_));
    CS_CUDA(cudaMemsetAsync(w->err, 0, sizeof(unsigned), cs_));
    CS_CUDA(cudaStreamSynchronize(cs_));
    if (e & kErrTimeout) {
        g_err = "a bounded device-side wait ran out";
        return CS_ERR_TIMEOUT;
    }
    if (e & kErrBounds) {
        g_err = "a device-side index check failed (CS_DEBUG build); the access was kept in bounds and the outputs "
                "are not valid";
        return CS_ERR_BOUNDS;
    }
    if (e & kErrInvalidQuery) {
        g_err = "invalid query rows (non-finite value, non-positive radius/axis or n_sigma < 0)";
        return CS_ERR_INVALID_ARG;
    }
    return CS_OK;
}

int32_t cs_tile_configs(int32_t *ids, int32_t cap) {
    if (!ids) cap = 0;
    return tile_configs(ids, cap);
}

cs_status cs_selftest_wait_timeout(int64_t spins, void *stream) {
    if (spins < 0) return invalid("spins must be >= 0");
    unsigned *err = nullptr;
    CS_CUDA(cudaMalloc(&err, sizeof(unsigned)));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = run_wait_selftest((long long)spins, err, s);
    unsigned h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    if (h & kErrTimeout) {
        g_err = "wait gave up as expected";
        return CS_ERR_TIMEOUT;
    }
    return CS_OK;
}

cs_status cs_release_scratch(void) {
    {
        std::lock_guard<std::mutex> lk(g_ws_mu);
        for (auto &kv : g_ws) free_ws(kv.second);
        g_ws.clear();
    }
    trim_temp_pools();
    return CS_OK;
}

int64_t cs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char *cs_last_error(void) { return g_err.c_str(); }

const char *cs_version(void) { return kDebugBuild ? "cs_b300 1.5 (sm_103a, CS_DEBUG)" : "cs_b300 1.5 (sm_103a)"; }

}  // extern "C"
