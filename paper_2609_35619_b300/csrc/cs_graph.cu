// cs_graph.cu -- captured query graphs and the tile autotuner.
//
// A query graph is one cs_query / cs_query_grad call (key sort, record
// preparation, fused cull+evaluate+reduce kernel, group epilogue) captured
// into a CUDA graph with private scratch, so a caller that repeats one query
// shape pays one graph launch instead of the ~20 kernel launches of the call.
// The autotuner times the fused kernel over every tile shape on the caller's
// own batch and records the fastest per (scene, primitive type, metric mode,
// batch-size class).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

// Autotuner log (cs_autotune_log): the file every cs_autotune call appends
// one JSON line to, or empty.
static std::mutex g_tune_log_mu;
static std::string g_tune_log;

static void append_tune_log(const Scene *sc, int prim_type, const cs_params &p, int64_t Q, int S, int reps,
                            const int32_t *ids, const float *times, int n, int32_t best) {
    std::lock_guard<std::mutex> lk(g_tune_log_mu);
    if (g_tune_log.empty()) return;
    FILE *f = fopen(g_tune_log.c_str(), "a");
    if (!f) return;
    fprintf(f, "{\"n_gaussians\": %lld, \"prim_type\": %d, \"mode\": %d, \"exact_variance\": %d, "
               "\"rows\": %lld, \"sweep\": %d, \"launch_rows\": %lld, \"reps\": %d, \"ms\": {",
            (long long)sc->n_kept, prim_type, (int)p.mode, (int)p.exact_variance, (long long)Q, S,
            (long long)(Q * S), reps);
    for (int i = 0; i < n; ++i) fprintf(f, "%s\"%d\": %.6f", i ? ", " : "", (int)ids[i], (double)times[i]);
    fprintf(f, "}, \"best\": %d}\n", (int)best);
    fclose(f);
}

constexpr uint32_t kGraphMagic = 0xC5B300A7u;

struct Graph {
    uint32_t magic = 0;
    cudaStream_t capture = nullptr;  // private stream the call was captured on
    Workspace *ws = nullptr;         // private scratch baked into the graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;             // kernels per launch
};

static void free_graph(Graph *g) {
    if (!g) return;
    g->magic = 0;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->ws) delete_workspace(g->ws);
    if (g->capture) cudaStreamDestroy(g->capture);
    delete g;
}

static cs_status check_graph(const cs_graph *h) {
    const Graph *g = reinterpret_cast<const Graph *>(h);
    if (!g || g->magic != kGraphMagic) {
        set_error("invalid graph handle");
        return CS_ERR_BAD_HANDLE;
    }
    return CS_OK;
}

// Capture `enqueue(stream, workspace)` on a private stream with private
// scratch (already grown by `reserve`) into an instantiated graph.
template <class Reserve, class Enqueue>
static cs_status capture_graph(Reserve reserve, Enqueue enqueue, cs_graph **out) {
    Graph *g = new Graph();
    cudaError_t e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "cudaStreamCreateWithFlags");
    }
    cs_status st;
    if ((st = new_workspace(g->capture, &g->ws)) != CS_OK || (st = reserve(g->ws)) != CS_OK) {
        free_graph(g);
        return st;
    }
    // the scratch is ready and argument errors surface before anything is captured
    e = cudaStreamSynchronize(g->capture);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "cudaStreamSynchronize");
    }
    const int64_t k0 = launch_total();
    e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    st = enqueue(g->capture, g->ws);
    const int64_t k1 = launch_total();
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(g->capture, &graph);
    g->graph = graph;
    if (st != CS_OK) {
        free_graph(g);
        return st;
    }
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        free_graph(g);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    // launches counted while capturing were not run; a replay counts them
    count_launches((int)(-(k1 - k0)));
    g->kernels = k1 - k0;
    g->magic = kGraphMagic;
    *out = reinterpret_cast<cs_graph *>(g);
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_graph_create(const cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                          float conservatism, float *out_metric, uint8_t *out_collide,
                          const float *grad_out, float *grad_centres, const cs_params *params,
                          cs_graph **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("a query graph takes device buffers only (host_io must be 0)");
    if (Q <= 0) return invalid("a query graph needs Q > 0");
    const bool grad = grad_centres != nullptr;
    if (grad && (out_metric || out_collide))
        return invalid("an adjoint graph takes grad_centres only (out_metric, out_collide NULL)");
    p.eval_events[0] = p.eval_events[1] = nullptr;
    if ((st = check_params(p)) != CS_OK) return st;
    const int S = sweep_blocks(p);
    return capture_graph([&](Workspace *w) {
                             cs_status r = grow_workspace(w, (size_t)Q, false);
                             return (r != CS_OK || S == 1) ? r : sweep_reserve(w, Q, prim_type, S);
                         },
                         [&](cudaStream_t s, Workspace *w) {
                             p.stream = s;
                             return query_common(scene, prim_type, prims, Q, conservatism, &p, grad, out_metric,
                                                 out_collide, grad_out, grad_centres, w);
                         },
                         out);
}

cs_status cs_mppi_graph_create(const cs_scene *scene, const cs_mppi_desc *desc, const float *x0, const float *U,
                               const float *eps, float *U_out, float *cost, float *weights, uint8_t *collide,
                               const cs_params *params, cs_graph **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    cs_status st = mppi_check(scene, desc, x0, U, eps, U_out);
    if (st != CS_OK) return st;
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("an MPPI graph takes device buffers only (host_io must be 0)");
    p.eval_events[0] = p.eval_events[1] = nullptr;
    return capture_graph([&](Workspace *w) { return mppi_reserve(w, desc->K, desc->T); },
                         [&](cudaStream_t s, Workspace *w) {
                             p.stream = s;
                             return mppi_common(scene, desc, x0, U, eps, U_out, cost, weights, collide, &p, w);
                         },
                         out);
}

cs_status cs_rrt_graph_create(const cs_scene *scene, const cs_rrt_desc *desc, float *nodes, int32_t *parent,
                              int32_t *count, const float *samples, int32_t *nearest, uint8_t *edge_free,
                              const cs_params *params, cs_graph **out) {
    if (!out) return invalid("out is NULL");
    *out = nullptr;
    cs_status st = rrt_check(scene, desc, nodes, parent, count, samples);
    if (st != CS_OK) return st;
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("an RRT graph takes device buffers only (host_io must be 0)");
    if ((st = check_params(p)) != CS_OK) return st;
    p.eval_events[0] = p.eval_events[1] = nullptr;
    return capture_graph([&](Workspace *w) { return rrt_reserve(w, desc->B, desc->M); },
                         [&](cudaStream_t s, Workspace *w) {
                             p.stream = s;
                             return rrt_common(scene, desc, nodes, parent, count, samples, nearest, edge_free, &p, w);
                         },
                         out);
}

cs_status cs_graph_launch(cs_graph *h, void *stream) {
    cs_status st = check_graph(h);
    if (st != CS_OK) return st;
    Graph *g = reinterpret_cast<Graph *>(h);
    CS_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    count_launches((int)g->kernels);
    return CS_OK;
}

cs_status cs_graph_sync(cs_graph *h, void *stream) {
    cs_status st = check_graph(h);
    if (st != CS_OK) return st;
    Graph *g = reinterpret_cast<Graph *>(h);
    cudaStream_t s = (cudaStream_t)stream;
    CS_CUDA(cudaStreamSynchronize(s));
    unsigned e = 0;
    CS_CUDA(cudaMemcpyAsync(&e, g->ws->err, sizeof(e), cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaMemsetAsync(g->ws->err, 0, sizeof(unsigned), s));
    CS_CUDA(cudaStreamSynchronize(s));
    if (e & kErrTimeout) {
        set_error("a bounded device-side wait ran out");
        return CS_ERR_TIMEOUT;
    }
    if (e & kErrInvalidQuery) {
        set_error("invalid query rows (non-finite value, non-positive radius/axis or n_sigma < 0)");
        return CS_ERR_INVALID_ARG;
    }
    return CS_OK;
}

int64_t cs_graph_kernels(const cs_graph *h) {
    if (check_graph(h) != CS_OK) return -1;
    return reinterpret_cast<const Graph *>(h)->kernels;
}

cs_status cs_graph_destroy(cs_graph *h) {
    if (!h) return CS_OK;
    cs_status st = check_graph(h);
    if (st != CS_OK) return st;
    free_graph(reinterpret_cast<Graph *>(h));
    return CS_OK;
}

cs_status cs_autotune(cs_scene *scene, int32_t prim_type, const float *prims, int64_t Q,
                      float conservatism, const cs_params *params, int32_t reps, int32_t *best,
                      float *ms, int32_t cap) {
    NvtxRange range("cs.autotune");
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!best) return invalid("best is NULL");
    if (reps < 1) return invalid("reps must be >= 1");
    if (Q <= 0) return invalid("autotuning needs Q > 0");
    Scene *sc = reinterpret_cast<Scene *>(scene);
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("cs_autotune takes device buffers only (host_io must be 0)");
    if ((st = check_params(p)) != CS_OK) return st;
    cudaStream_t s = (cudaStream_t)p.stream;
    Workspace *ws = nullptr;
    if ((st = get_workspace(sc->device, s, (size_t)Q, false, &ws)) != CS_OK) return st;
    // a sweep's scratch first: the per-row output below must not move afterwards
    const int S = sweep_blocks(p);
    if (S > 1 && (st = sweep_reserve(ws, Q, prim_type, S)) != CS_OK) return st;
    // timed launches write to scratch only: per-row metric, no groups
    p.group_size = 0;
    p.out_count = nullptr;
    p.out_group_metric = nullptr;
    p.out_group_collide = nullptr;
    p.out_pair_stats = nullptr;
    p.out_kernel_stats = nullptr;
    cudaEvent_t ev[2];
    CS_CUDA(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(cudaErrorUnknown, "cudaEventCreate");
    }
    int32_t ids[64];
    float times[64];
    const int n = tile_configs(ids, 64);
    float best_ms = INFINITY;
    int32_t best_id = 0;
    for (int i = 0; i < n && st == CS_OK; ++i) {
        p.tile_config = ids[i];
        double total = 0.0;
        for (int r = 0; r <= reps && st == CS_OK; ++r) {
            p.eval_events[0] = ev[0];
            p.eval_events[1] = ev[1];
            st = query_common(scene, prim_type, prims, Q, conservatism, &p, false, ws->io_metric,
                              nullptr, nullptr, nullptr, ws);
            if (st != CS_OK) break;
            cudaError_t e = cudaEventSynchronize(ev[1]);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "autotune timing");
                break;
            }
            if (r > 0) total += t;  // launch 0 warms up
        }
        if (st != CS_OK) break;
        const float mean = (float)(total / reps);
        times[i] = mean;
        if (ms && i < cap) ms[i] = mean;
        if (mean < best_ms) {
            best_ms = mean;
            best_id = ids[i];
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != CS_OK) return st;
    {
        std::lock_guard<std::mutex> lk(sc->tune_mu);
        sc->tuned[tune_key(prim_type, p.mode, Q * S)] = best_id;  // keyed by the launch's rows
    }
    append_tune_log(sc, prim_type, p, Q, S, reps, ids, times, n, best_id);
    *best = best_id;
    return CS_OK;
}

cs_status cs_autotune_log(const char *path) {
    std::lock_guard<std::mutex> lk(g_tune_log_mu);
    g_tune_log = path ? path : "";
    return CS_OK;
}

}  // extern "C"
