// cs_mppi.cu -- one MPPI iteration with the collision cost of Section II-D,
// fused on the device: rollouts of the sampled control sequences, the
// conservative metric of every rollout position (the query path, mean cost
// per position summed over the horizon), the per-rollout cost, the Eq. 10
// softmin weights and the update of the nominal sequence.
//
// The robot is one sphere under single-integrator (velocity) control:
//   u[k,t] = U[t] + eps[k,t],  x[k,t+1] = x[k,t] + dt u[k,t],  x[k,0] = x0,
// and rollout k is scored by
//   C^k = w_col sum_t mean-cost(x[k,t+1]) + w_goal sum_t |x[k,t+1] - g|^2
//         + w_term |x[k,T] - g|^2 + w_u sum_t |u[k,t]|^2,
// the paper's cost sum with the image term left out (no image model here).
#include <cuda_runtime.h>

#include <math.h>

#include "cs_internal.cuh"

namespace cs {

namespace {

struct MppiConsts {
    int K, T;
    float dt, radius;
    float w_collision, w_goal, w_terminal, w_control, lambda;
    float gx, gy, gz;
};

constexpr int kWeightThreads = 1024;

// One thread per rollout: integrate, write the sphere of every step, and the
// task + control part of the cost (accumulated in step order).
__global__ void k_mppi_rollout(const float *__restrict__ x0, const float *__restrict__ U,
                               const float *__restrict__ eps, MppiConsts c, float4 *__restrict__ spheres,
                               float *__restrict__ tc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= c.K) return;
    float x = x0[0], y = x0[1], z = x0[2];
    float task = 0.f, ctrl = 0.f;
    const float *e = eps + (size_t)k * c.T * 3;
    for (int t = 0; t < c.T; ++t) {
        const float ux = U[3 * t] + e[3 * t], uy = U[3 * t + 1] + e[3 * t + 1], uz = U[3 * t + 2] + e[3 * t + 2];
        x = fmaf(c.dt, ux, x);
        y = fmaf(c.dt, uy, y);
        z = fmaf(c.dt, uz, z);
        spheres[(size_t)k * c.T + t] = make_float4(x, y, z, c.radius);
        const float dx = x - c.gx, dy = y - c.gy, dz = z - c.gz;
        task += dx * dx + dy * dy + dz * dz;
        ctrl += ux * ux + uy * uy + uz * uz;
    }
    const float dx = x - c.gx, dy = y - c.gy, dz = z - c.gz;
    tc[k] = c.w_goal * task + c.w_terminal * (dx * dx + dy * dy + dz * dz) + c.w_control * ctrl;
}

// One block: C^k, then Eq. 10 as exp(-(C^k - min C) / lambda) over its sum.
// Each thread reduces rollouts thread, thread + 1024, ... in order, then a
// fixed tree: the bits do not depend on anything but K.
__global__ void __launch_bounds__(kWeightThreads) k_mppi_weights(const float *__restrict__ col,
                                                                 const float *__restrict__ tc, MppiConsts c,
                                                                 float *__restrict__ cost, float *__restrict__ w) {
    __shared__ float red[kWeightThreads];
    const int tid = threadIdx.x;
    float mn = INFINITY;
    for (int k = tid; k < c.K; k += kWeightThreads) {
        const float C = fmaf(c.w_collision, col[k], tc[k]);
        cost[k] = C;
        mn = fminf(mn, C);
    }
    red[tid] = mn;
    __syncthreads();
    for (int o = kWeightThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] = fminf(red[tid], red[tid + o]);
        __syncthreads();
    }
    mn = red[0];
    __syncthreads();
    float sum = 0.f;
    for (int k = tid; k < c.K; k += kWeightThreads) {
        const float e = expf((mn - cost[k]) / c.lambda);
        w[k] = e;
        sum += e;
    }
    red[tid] = sum;
    __syncthreads();
    for (int o = kWeightThreads / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const float inv = 1.f / red[0];
    for (int k = tid; k < c.K; k += kWeightThreads) w[k] *= inv;
}

// U_out[t,d] = U[t,d] + sum_k w[k] eps[k,t,d]: one warp per (t, d), lane l
// summing rollouts l, l + 32, ... in order, then a fixed xor tree.
__global__ void k_mppi_update(const float *__restrict__ U, const float *__restrict__ eps,
                              const float *__restrict__ w, MppiConsts c, float *__restrict__ U_out) {
    const int o = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= c.T * 3) return;  // whole warps leave together
    float s = 0.f;
    for (int k = lane; k < c.K; k += 32) s = fmaf(w[k], eps[(size_t)k * c.T * 3 + o], s);
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
    if (lane == 0) U_out[o] = U[o] + s;
}

}  // namespace

cs_status mppi_check(const cs_scene *scene, const cs_mppi_desc *d, const float *x0, const float *U,
                     const float *eps, const float *U_out) {
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!d) return invalid("desc is NULL");
    if (d->K < 1 || d->K > (1 << 20)) return invalid("K must lie in [1, 2^20]");
    if (d->T < 1 || d->T > 1024) return invalid("T must lie in [1, 1024]");
    if ((int64_t)d->K * d->T > ((int64_t)1 << 26)) return invalid("K * T must not exceed 2^26");
    if (!(d->dt > 0.f) || !isfinite(d->dt)) return invalid("dt must be finite and > 0");
    if (!(d->radius > 0.f) || !isfinite(d->radius)) return invalid("radius must be finite and > 0");
    if (!(d->nsigma >= 0.f) || !isfinite(d->nsigma)) return invalid("nsigma must be finite and >= 0");
    if (!(d->lambda > 0.f) || !isfinite(d->lambda)) return invalid("lambda must be finite and > 0");
    const float ws[4] = {d->w_collision, d->w_goal, d->w_terminal, d->w_control};
    for (float v : ws)
        if (!(v >= 0.f) || !isfinite(v)) return invalid("cost weights must be finite and >= 0");
    for (int a = 0; a < 3; ++a)
        if (!isfinite(d->goal[a])) return invalid("goal must be finite");
    if (!x0 || !U || !eps || !U_out) return invalid("x0, U, eps and U_out are required");
    return CS_OK;
}

// Pooled (or owned) scratch of an iteration of K rollouts x T steps, grown
// before use so that a captured iteration allocates nothing.
cs_status mppi_reserve(Workspace *w, int64_t K, int64_t T) {
    cs_status st = grow_workspace(w, (size_t)(K * T), false);
    if (st != CS_OK) return st;
    const size_t need = 4 * (size_t)(K * T) + 4 * (size_t)K;
    if (w->cap_mppi < need) {
        if (w->mppi) CS_CUDA(cudaFree(w->mppi));
        w->mppi = nullptr;
        w->cap_mppi = 0;
        CS_CUDA(cudaMalloc(&w->mppi, 4 * need));
        w->cap_mppi = need;
    }
    return CS_OK;
}

cs_status mppi_common(const cs_scene *scene, const cs_mppi_desc *d, const float *x0, const float *U,
                      const float *eps, float *U_out, float *cost, float *weights, uint8_t *collide,
                      const cs_params *params, Workspace *own_ws) {
    cs_status st = mppi_check(scene, d, x0, U, eps, U_out);
    if (st != CS_OK) return st;
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("cs_mppi_step takes device buffers only (host_io must be 0)");
    if ((st = check_params(p)) != CS_OK) return st;
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    cudaStream_t s = (cudaStream_t)p.stream;
    const int64_t Q = (int64_t)d->K * d->T;

    // scratch: spheres [Q,4], collision cost [K], task + control [K], cost [K], weights [K]
    Workspace *w = own_ws;
    if (!w && (st = get_workspace(sc->device, s, (size_t)Q, false, &w)) != CS_OK) return st;
    if ((st = mppi_reserve(w, d->K, d->T)) != CS_OK) return st;
    float4 *spheres = reinterpret_cast<float4 *>(w->mppi);
    float *col = w->mppi + 4 * Q, *tc = col + d->K;
    float *c_out = cost ? cost : tc + d->K, *w_out = weights ? weights : c_out + d->K;

    MppiConsts c;
    c.K = d->K;
    c.T = d->T;
    c.dt = d->dt;
    c.radius = d->radius;
    c.w_collision = d->w_collision;
    c.w_goal = d->w_goal;
    c.w_terminal = d->w_terminal;
    c.w_control = d->w_control;
    c.lambda = d->lambda;
    c.gx = d->goal[0];
    c.gy = d->goal[1];
    c.gz = d->goal[2];

    k_mppi_rollout<<<(c.K + 127) / 128, 128, 0, s>>>(x0, U, eps, c, spheres, tc);
    count_launches(1);
    CS_CUDA(cudaGetLastError());
    // the metric of every rollout position, mean cost per position (Eq. 11
    // averaged over the neighbour set) summed over the horizon per rollout
    cs_params q = p;
    q.mode = CS_METRIC_MEAN_COST;
    q.group_size = d->T;
    q.nsigma_per_query = nullptr;
    q.out_count = nullptr;
    q.out_group_metric = col;
    q.out_group_collide = collide;
    q.host_io = 0;
    if ((st = query_common(scene, CS_PRIM_SPHERE, reinterpret_cast<const float *>(spheres), Q, d->nsigma, &q,
                           false, nullptr, nullptr, nullptr, nullptr, w)) != CS_OK)
        return st;
    k_mppi_weights<<<1, kWeightThreads, 0, s>>>(col, tc, c, c_out, w_out);
    k_mppi_update<<<(c.T * 3 * 32 + 255) / 256, 256, 0, s>>>(U, eps, w_out, c, U_out);
    count_launches(2);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_mppi_step(const cs_scene *scene, const cs_mppi_desc *desc, const float *x0, const float *U,
                       const float *eps, float *U_out, float *cost, float *weights, uint8_t *collide,
                       const cs_params *params) {
    return mppi_common(scene, desc, x0, U, eps, U_out, cost, weights, collide, params, nullptr);
}

}  // extern "C"
