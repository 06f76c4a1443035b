// cs_serve.cu -- the serving loop: resident scenes, continuous batching of
// uneven collision-query requests, per-request latency.
//
// The paper has no counterpart; this is the runtime around the query path.
// A server owns `slots` batch slots.  Each slot has its own stream, private
// query scratch and fixed device / pinned host buffers for `slot_rows` rows,
// all allocated when the server is created, so admission is by memory: a
// request waits until a slot is free, then joins that slot's batch with the
// other waiting requests for the same scene and primitive type, as far as
// the slot's rows and request count allow.  A launcher thread forms a batch
// as soon as a slot is free and requests wait, so batches formed while
// others run overlap on the device (continuous batching).  A batch is one
// pass of the query path over the concatenated rows with per-row n_sigma,
// plus a segmented group epilogue; per-row results do not depend on which
// rows share a launch (the fused kernel's reductions run in a fixed order
// per primitive), so a request's results equal those of a cs_query call on
// it alone.  Completion runs as a host function on the slot's stream after
// the results have been copied back: it scatters each request's rows to the
// caller's buffers, stamps the completion time and frees the slot.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

// Group outputs of the requests of one batch: segment s covers batch rows
// [row, row + rows) reduced in runs of G into group outputs [out, out +
// ceil(rows / G)).  One warp per group output; each group is reduced in the
// order k_group uses for its size, so the bits equal a cs_query call.
struct GroupSeg {
    int32_t row, rows, G, out;
};

__global__ void k_group_segments(const float *__restrict__ metric, const uint8_t *__restrict__ collide,
                                 const GroupSeg *__restrict__ segs, int nseg, int ngroups,
                                 float *__restrict__ gm, uint8_t *__restrict__ gc) {
    const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= ngroups) return;  // whole warps leave together
    int lo = 0, hi = nseg - 1;  // last segment with out <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].out <= g) lo = mid;
        else hi = mid - 1;
    }
    const GroupSeg sg = segs[lo];
    const int b = sg.row + (g - sg.out) * sg.G, e = min(sg.row + sg.rows, b + sg.G);
    float s;
    unsigned c;
    if (sg.G >= kGroupWarpMin) {
        group_rows_warp(metric, collide, b, e, lane, s, c);
    } else {
        if (lane != 0) return;
        group_rows_serial(metric, collide, b, e, s, c);
    }
    if (lane == 0) {
        gm[g] = s;
        gc[g] = (uint8_t)c;
    }
}

constexpr uint32_t kServerMagic = 0xC5B300A5u;

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    cs_request r;
    uint64_t ticket = 0;
    double submitted = 0, launched = 0, completed = 0;
    int64_t batch_rows = 0, batch_requests = 0;
    int32_t status = CS_OK;
    bool done = false;
};

struct Server;

struct Slot {
    Server *srv = nullptr;
    int index = 0;
    cudaStream_t stream = nullptr;
    Workspace *ws = nullptr;
    // device
    float *d_prims = nullptr, *d_ns = nullptr, *d_metric = nullptr, *d_gm = nullptr;
    uint8_t *d_collide = nullptr, *d_gc = nullptr;
    int32_t *d_count = nullptr;
    GroupSeg *d_segs = nullptr;
    // pinned host
    float *h_prims = nullptr, *h_ns = nullptr, *h_metric = nullptr, *h_gm = nullptr;
    uint8_t *h_collide = nullptr, *h_gc = nullptr;
    int32_t *h_count = nullptr;
    GroupSeg *h_segs = nullptr;
    unsigned *h_err = nullptr;
    // the batch in flight
    bool busy = false;
    std::vector<Request *> reqs;
    std::vector<int64_t> row0, grp0;  // first batch row / group output of each request
    int64_t rows = 0;
    bool want_count = false;
    // captured query graphs by (scene, primitive type, counts, bucket)
    std::unordered_map<uint64_t, cudaGraphExec_t> graphs;
};

struct Server {
    uint32_t magic = 0;
    std::vector<Scene *> scenes;
    cs_server_config cfg;
    int device = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_launch;  // pending work or a free slot or stop
    std::condition_variable cv_done;    // a request completed
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> live;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread launcher;
    // statistics
    int64_t n_batches = 0, n_rows = 0, n_requests = 0, max_batch_rows = 0, max_batch_requests = 0;
    std::string thread_error;
};

static void free_slot(Slot &s) {
    for (auto &kv : s.graphs) cudaGraphExecDestroy(kv.second);
    s.graphs.clear();
    void *dev[] = {s.d_prims, s.d_ns, s.d_metric, s.d_gm, s.d_collide, s.d_gc, s.d_count, s.d_segs};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *host[] = {s.h_prims, s.h_ns, s.h_metric, s.h_gm, s.h_collide, s.h_gc, s.h_count, s.h_segs, s.h_err};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    if (s.ws) delete_workspace(s.ws);
    if (s.stream) cudaStreamDestroy(s.stream);
    s = Slot();
}

static cs_status alloc_slot(Slot &s, int64_t rows, int32_t max_req) {
    const size_t R = (size_t)rows;
    CS_CUDA(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    cs_status st = new_workspace(s.stream, &s.ws);
    if (st != CS_OK) return st;
    if ((st = grow_workspace(s.ws, R, false)) != CS_OK) return st;
    CS_CUDA(cudaMalloc(&s.d_prims, 40 * R));
    CS_CUDA(cudaMalloc(&s.d_ns, 4 * R));
    CS_CUDA(cudaMalloc(&s.d_metric, 4 * R));
    CS_CUDA(cudaMalloc(&s.d_gm, 4 * R));
    CS_CUDA(cudaMalloc(&s.d_collide, R));
    CS_CUDA(cudaMalloc(&s.d_gc, R));
    CS_CUDA(cudaMalloc(&s.d_count, 4 * R));
    CS_CUDA(cudaMalloc(&s.d_segs, sizeof(GroupSeg) * (size_t)max_req));
    CS_CUDA(cudaHostAlloc(&s.h_prims, 40 * R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_ns, 4 * R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_metric, 4 * R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_gm, 4 * R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_collide, R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_gc, R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_count, 4 * R, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_segs, sizeof(GroupSeg) * (size_t)max_req, cudaHostAllocDefault));
    CS_CUDA(cudaHostAlloc(&s.h_err, sizeof(unsigned), cudaHostAllocDefault));
    s.reqs.reserve((size_t)max_req);
    s.row0.reserve((size_t)max_req);
    s.grp0.reserve((size_t)max_req);
    return CS_OK;
}

static int stride_of(int32_t prim_type) { return prim_type == CS_PRIM_SPHERE ? 4 : 10; }

// Host function on the slot's stream, after the results are in pinned
// memory: scatter them to the callers' buffers and free the slot.  Calls no
// CUDA API.
static void CUDART_CB on_batch_done(void *arg) {
    Slot *s = static_cast<Slot *>(arg);
    Server *srv = s->srv;
    const double t = now_s();
    const unsigned err = *s->h_err;
    const int32_t status = (err & kErrTimeout) ? CS_ERR_TIMEOUT : (err & kErrInvalidQuery) ? CS_ERR_INVALID_ARG : CS_OK;
    for (size_t i = 0; i < s->reqs.size(); ++i) {
        Request *q = s->reqs[i];
        const cs_request &r = q->r;
        const int64_t b = s->row0[i];
        if (r.out_metric) memcpy(r.out_metric, s->h_metric + b, 4 * (size_t)r.Q);
        if (r.out_collide) memcpy(r.out_collide, s->h_collide + b, (size_t)r.Q);
        if (r.out_count) memcpy(r.out_count, s->h_count + b, 4 * (size_t)r.Q);
        if (r.group_size > 0) {
            const int64_t ng = (r.Q + r.group_size - 1) / r.group_size;
            if (r.out_group_metric) memcpy(r.out_group_metric, s->h_gm + s->grp0[i], 4 * (size_t)ng);
            if (r.out_group_collide) memcpy(r.out_group_collide, s->h_gc + s->grp0[i], (size_t)ng);
        }
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (Request *q : s->reqs) {
            q->completed = t;
            q->status = status;
            q->done = true;
        }
        s->reqs.clear();
        s->busy = false;
    }
    srv->cv_done.notify_all();
    srv->cv_launch.notify_all();
}

// Rows of the graph a batch of `rows` rows replays: the next power of two
// from 1024, at most the slot's rows.
static int64_t graph_bucket(int64_t rows, int64_t slot_rows) {
    int64_t b = 1024;
    while (b < rows) b <<= 1;
    return std::min(b, slot_rows);
}

// The query path of a batch as one graph replay.  The batch's rows are
// already in pinned memory; rows [rows, bucket) are padded with primitives
// far outside every scene (valid rows whose reach meets no chunk: count 0,
// metric 0, flag 0), which sort after the real rows and change none of
// their results.  The padded rows are copied up with the batch; the graph
// for (scene, primitive type, counts wanted, bucket) is captured on the
// slot's stream the first time it is needed.
static cs_status run_graph(Server *srv, Slot &s, int32_t scene, int32_t prim, int64_t rows, const cs_params &p,
                           cudaError_t &e) {
    const int64_t bucket = graph_bucket(rows, srv->cfg.slot_rows);
    const int stride = stride_of(prim);
    for (int64_t r = rows; r < bucket; ++r) {
        float *q = s.h_prims + r * stride;
        q[0] = q[1] = q[2] = 1e30f;
        if (stride == 4) {
            q[3] = 1.f;
        } else {
            q[3] = 1.f; q[4] = q[5] = q[6] = 0.f;
            q[7] = q[8] = q[9] = 1.f;
        }
        s.h_ns[r] = 0.f;
    }
    cudaStream_t st = s.stream;
    if (bucket > rows) {
        e = cudaMemcpyAsync(s.d_prims + rows * stride, s.h_prims + rows * stride,
                            4 * (size_t)stride * (size_t)(bucket - rows), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.d_ns + rows, s.h_ns + rows, 4 * (size_t)(bucket - rows), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return CS_ERR_CUDA;
    }
    const uint64_t key = ((uint64_t)scene << 40) | ((uint64_t)prim << 36) | ((uint64_t)(p.out_count != nullptr) << 35) |
                         (uint64_t)bucket;
    auto it = s.graphs.find(key);
    if (it == s.graphs.end()) {
        // the slot's stream is idle here (the slot was free); capture the query path once
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return CS_ERR_CUDA;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return CS_ERR_CUDA;
        const cs_status cst = query_common(reinterpret_cast<cs_scene *>(srv->scenes[scene]), prim, s.d_prims, bucket,
                                           0.f, &p, false, s.d_metric, s.d_collide, nullptr, nullptr, s.ws);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (cst != CS_OK) {
            if (g) cudaGraphDestroy(g);
            return cst;
        }
        if (e != cudaSuccess) return CS_ERR_CUDA;
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return CS_ERR_CUDA;
        it = s.graphs.emplace(key, ex).first;
    }
    e = cudaGraphLaunch(it->second, st);
    return e == cudaSuccess ? CS_OK : CS_ERR_CUDA;
}

// Form and launch one batch on slot `s` from the pending queue (lock held on
// entry, released while the batch is assembled and enqueued).
static void launch_batch(Server *srv, Slot &s, std::unique_lock<std::mutex> &lk) {
    NvtxRange range("cs.serve.batch");
    const int32_t scene = srv->pending.front()->r.scene, prim = srv->pending.front()->r.prim_type;
    const int64_t cap = srv->cfg.slot_rows;
    int64_t rows = 0;
    s.reqs.clear();
    for (auto it = srv->pending.begin(); it != srv->pending.end();) {
        Request *q = *it;
        if ((int32_t)s.reqs.size() >= srv->cfg.max_requests) break;
        if (q->r.scene == scene && q->r.prim_type == prim) {
            if (rows + q->r.Q > cap) break;  // FIFO within a key: no overtaking
            rows += q->r.Q;
            s.reqs.push_back(q);
            it = srv->pending.erase(it);
        } else {
            ++it;
        }
    }
    s.busy = true;
    s.rows = rows;
    srv->n_batches += 1;
    srv->n_rows += rows;
    srv->n_requests += (int64_t)s.reqs.size();
    srv->max_batch_rows = std::max(srv->max_batch_rows, rows);
    srv->max_batch_requests = std::max(srv->max_batch_requests, (int64_t)s.reqs.size());
    lk.unlock();

    // assemble the batch in pinned memory
    const int stride = stride_of(prim);
    const double t_launch = now_s();
    int64_t r0 = 0, g0 = 0;
    int nseg = 0;
    s.row0.clear();
    s.grp0.clear();
    s.want_count = false;
    for (Request *q : s.reqs) {
        const cs_request &r = q->r;
        memcpy(s.h_prims + r0 * stride, r.prims, 4 * (size_t)stride * (size_t)r.Q);
        std::fill(s.h_ns + r0, s.h_ns + r0 + r.Q, r.conservatism);
        s.row0.push_back(r0);
        s.grp0.push_back(g0);
        if (r.group_size > 0) {
            s.h_segs[nseg++] = GroupSeg{(int32_t)r0, (int32_t)r.Q, r.group_size, (int32_t)g0};
            g0 += (r.Q + r.group_size - 1) / r.group_size;
        }
        s.want_count |= r.out_count != nullptr;
        q->launched = t_launch;
        q->batch_rows = rows;
        q->batch_requests = (int64_t)s.reqs.size();
        r0 += r.Q;
    }
    cs_params p = srv->cfg.params;
    p.stream = s.stream;
    p.nsigma_per_query = s.d_ns;
    p.group_size = 0;
    p.host_io = 0;
    p.out_count = s.want_count ? s.d_count : nullptr;
    p.out_group_metric = nullptr;
    p.out_group_collide = nullptr;
    p.out_pair_stats = nullptr;
    p.out_kernel_stats = nullptr;
    p.eval_events[0] = p.eval_events[1] = nullptr;
    p.tile_config = srv->cfg.tile_config;
    cudaStream_t st = s.stream;
    cudaError_t e = cudaSuccess;
    cs_status cst = CS_OK;
    auto ok = [&]() { return e == cudaSuccess && cst == CS_OK; };
    e = cudaMemsetAsync(s.ws->err, 0, sizeof(unsigned), st);
    if (ok()) e = cudaMemcpyAsync(s.d_prims, s.h_prims, 4 * (size_t)stride * (size_t)rows, cudaMemcpyHostToDevice, st);
    if (ok()) e = cudaMemcpyAsync(s.d_ns, s.h_ns, 4 * (size_t)rows, cudaMemcpyHostToDevice, st);
    if (ok() && nseg > 0) e = cudaMemcpyAsync(s.d_segs, s.h_segs, sizeof(GroupSeg) * nseg, cudaMemcpyHostToDevice, st);
    if (ok() && srv->cfg.use_graphs) {
        cst = run_graph(srv, s, scene, prim, rows, p, e);
    } else if (ok()) {
        cst = query_common(reinterpret_cast<cs_scene *>(srv->scenes[scene]), prim, s.d_prims, rows, 0.f, &p,
                           false, s.d_metric, s.d_collide, nullptr, nullptr, s.ws);
    }
    if (ok() && nseg > 0) {
        k_group_segments<<<(unsigned)((g0 * 32 + 255) / 256), 256, 0, st>>>(s.d_metric, s.d_collide, s.d_segs,
                                                                           nseg, (int)g0, s.d_gm, s.d_gc);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (ok()) e = cudaMemcpyAsync(s.h_metric, s.d_metric, 4 * (size_t)rows, cudaMemcpyDeviceToHost, st);
    if (ok()) e = cudaMemcpyAsync(s.h_collide, s.d_collide, (size_t)rows, cudaMemcpyDeviceToHost, st);
    if (ok() && s.want_count) e = cudaMemcpyAsync(s.h_count, s.d_count, 4 * (size_t)rows, cudaMemcpyDeviceToHost, st);
    if (ok() && g0 > 0) e = cudaMemcpyAsync(s.h_gm, s.d_gm, 4 * (size_t)g0, cudaMemcpyDeviceToHost, st);
    if (ok() && g0 > 0) e = cudaMemcpyAsync(s.h_gc, s.d_gc, (size_t)g0, cudaMemcpyDeviceToHost, st);
    if (ok()) e = cudaMemcpyAsync(s.h_err, s.ws->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (ok()) e = cudaLaunchHostFunc(st, on_batch_done, &s);
    lk.lock();
    if (!ok()) {
        // nothing will complete this batch: fail its requests now
        srv->thread_error = e != cudaSuccess ? std::string(cudaGetErrorString(e)) : std::string("query failed");
        cudaStreamSynchronize(st);
        const double t = now_s();
        for (Request *q : s.reqs) {
            q->status = e != cudaSuccess ? CS_ERR_CUDA : cst;
            q->completed = t;
            q->done = true;
        }
        s.reqs.clear();
        s.busy = false;
        srv->cv_done.notify_all();
    }
}

static void launcher_main(Server *srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        Slot *free_slot = nullptr;
        srv->cv_launch.wait(lk, [&] {
            if (srv->stop) return true;
            if (srv->pending.empty()) return false;
            for (Slot &s : srv->slots)
                if (!s.busy) {
                    free_slot = &s;
                    return true;
                }
            return false;
        });
        if (srv->stop) break;
        launch_batch(srv, *free_slot, lk);
    }
}

static cs_status check_server(const cs_server *h) {
    const Server *s = reinterpret_cast<const Server *>(h);
    if (!s || s->magic != kServerMagic) {
        set_error("invalid server handle");
        return CS_ERR_BAD_HANDLE;
    }
    return CS_OK;
}

static void destroy_server(Server *srv) {
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->magic = 0;
    }
    srv->cv_launch.notify_all();
    if (srv->launcher.joinable()) srv->launcher.join();
    for (Slot &s : srv->slots)
        if (s.stream) cudaStreamSynchronize(s.stream);
    for (auto &kv : srv->live) delete kv.second;
    for (Slot &s : srv->slots) free_slot(s);
    delete srv;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_server_config_init(cs_server_config *c) {
    if (!c) return invalid("config is NULL");
    memset(c, 0, sizeof(*c));
    c->slots = 3;
    c->slot_rows = 1 << 19;
    c->max_requests = 4096;
    c->tile_config = CS_TILE_TUNED;
    c->use_graphs = 1;
    return cs_params_init(&c->params);
}

cs_status cs_server_create(cs_scene *const *scenes, int32_t n_scenes, const cs_server_config *cfg,
                           cs_server **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    if (!scenes || n_scenes < 1) return invalid("at least one scene is required");
    cs_server_config c;
    if (cfg) c = *cfg;
    else cs_server_config_init(&c);
    if (c.slots < 1 || c.slots > 16) return invalid("slots must lie in [1, 16]");
    if (c.slot_rows < 1 || c.slot_rows > (1 << 28)) return invalid("slot_rows must lie in [1, 2^28]");
    if (c.max_requests < 1) return invalid("max_requests must be >= 1");
    cs_params p = c.params;
    p.tile_config = c.tile_config;
    cs_status st = check_params(p);
    if (st != CS_OK) return st;
    if (p.sweep_count >= 2) return invalid("the server takes no conservatism sweep (n_sigma is per request)");
    Server *srv = new Server();
    srv->cfg = c;
    for (int i = 0; i < n_scenes; ++i) {
        if ((st = check_scene(scenes[i])) != CS_OK) {
            delete srv;
            return st;
        }
        srv->scenes.push_back(reinterpret_cast<Scene *>(scenes[i]));
    }
    srv->device = srv->scenes[0]->device;
    for (Scene *sc : srv->scenes)
        if (sc->device != srv->device) {
            delete srv;
            return invalid("every scene of a server must live on one device");
        }
    srv->slots.resize((size_t)c.slots);
    for (int i = 0; i < c.slots; ++i) {
        srv->slots[i].srv = srv;
        srv->slots[i].index = i;
        if ((st = alloc_slot(srv->slots[i], c.slot_rows, c.max_requests)) != CS_OK) {
            for (Slot &s : srv->slots) free_slot(s);
            delete srv;
            return st;
        }
    }
    srv->magic = kServerMagic;
    srv->launcher = std::thread(launcher_main, srv);
    *out = reinterpret_cast<cs_server *>(srv);
    return CS_OK;
}

cs_status cs_server_submit(cs_server *h, const cs_request *req, uint64_t *ticket) {
    cs_status st = check_server(h);
    if (st != CS_OK) return st;
    Server *srv = reinterpret_cast<Server *>(h);
    if (!req || !ticket) return invalid("request or ticket is NULL");
    const cs_request &r = *req;
    if (r.scene < 0 || r.scene >= (int32_t)srv->scenes.size()) return invalid("scene index out of range");
    if (r.prim_type != CS_PRIM_SPHERE && r.prim_type != CS_PRIM_ELLIPSOID)
        return invalid("prim_type must be CS_PRIM_SPHERE or CS_PRIM_ELLIPSOID");
    if (r.Q < 1 || r.Q > srv->cfg.slot_rows) return invalid("Q must lie in [1, slot_rows]");
    if (!r.prims) return invalid("prims is NULL");
    if (!(r.conservatism >= 0.f) || !std::isfinite(r.conservatism))
        return invalid("conservatism (n_sigma) must be finite and >= 0");
    if (r.group_size < 0) return invalid("group_size must be >= 0");
    if (!r.out_metric && !r.out_collide && !r.out_count &&
        !(r.group_size > 0 && (r.out_group_metric || r.out_group_collide)))
        return invalid("no output requested");
    const int stride = stride_of(r.prim_type);
    for (int64_t j = 0; j < r.Q; ++j) {
        const float *x = r.prims + j * stride;
        for (int a = 0; a < stride; ++a)
            if (!std::isfinite(x[a])) return invalid("non-finite value in prims");
        if (r.prim_type == CS_PRIM_SPHERE ? !(x[3] > 0.f) : !(x[7] > 0.f && x[8] > 0.f && x[9] > 0.f))
            return invalid("non-positive radius or semi-axis in prims");
    }
    Request *q = new Request();
    q->r = r;
    q->submitted = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        q->ticket = srv->next_ticket++;
        srv->live[q->ticket] = q;
        srv->pending.push_back(q);
    }
    srv->cv_launch.notify_one();
    *ticket = q->ticket;
    return CS_OK;
}

cs_status cs_server_wait(cs_server *h, uint64_t ticket, double timeout_s, cs_request_times *times) {
    cs_status st = check_server(h);
    if (st != CS_OK) return st;
    Server *srv = reinterpret_cast<Server *>(h);
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->live.find(ticket);
    if (it == srv->live.end()) return invalid("unknown ticket (never issued or already waited for)");
    Request *q = it->second;
    const auto pred = [&] { return q->done; };
    if (timeout_s < 0) {
        srv->cv_done.wait(lk, pred);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        set_error("the request has not completed within the timeout");
        return CS_ERR_TIMEOUT;
    }
    if (times) {
        times->submitted = q->submitted;
        times->launched = q->launched;
        times->completed = q->completed;
        times->batch_rows = q->batch_rows;
        times->batch_requests = q->batch_requests;
        times->status = q->status;
    }
    const int32_t status = q->status;
    srv->live.erase(it);
    delete q;
    if (status != CS_OK) set_error("the request's batch failed: " + srv->thread_error);
    return (cs_status)status;
}

cs_status cs_server_stats_get(cs_server *h, cs_server_stats *out) {
    cs_status st = check_server(h);
    if (st != CS_OK) return st;
    if (!out) return invalid("out is NULL");
    Server *srv = reinterpret_cast<Server *>(h);
    std::lock_guard<std::mutex> lk(srv->mu);
    out->batches = srv->n_batches;
    out->rows = srv->n_rows;
    out->requests = srv->n_requests;
    out->max_batch_rows = srv->max_batch_rows;
    out->max_batch_requests = srv->max_batch_requests;
    out->pending = (int64_t)srv->pending.size();
    int64_t busy = 0;
    for (Slot &s : srv->slots) busy += s.busy ? 1 : 0;
    out->busy_slots = busy;
    return CS_OK;
}

double cs_server_clock(void) { return now_s(); }

cs_status cs_server_destroy(cs_server *h) {
    if (!h) return CS_OK;
    cs_status st = check_server(h);
    if (st != CS_OK) return st;
    destroy_server(reinterpret_cast<Server *>(h));
    return CS_OK;
}

}  // extern "C"
