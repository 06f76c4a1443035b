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
#include <string.h>

#include "cs_internal.cuh"

namespace cs {

namespace {

struct MppiConsts {
    int K, T;
    float dt, radius;
    float w_collision, w_goal, w_terminal, w_control, lambda;
    float gx, gy, gz;
    int fixed_ends;  // path refinement: the first and last rows of U stay
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
    const bool fixed = c.fixed_ends && (o < 3 || o >= 3 * (c.T - 1));
    if (lane == 0) U_out[o] = fixed ? U[o] : U[o] + s;
}

// Path refinement: one thread per (rollout, spline segment) writes the
// segment's M sample spheres (the stated float32 operation order); the
// rollout's last thread also writes the end point.
__global__ void k_refine_points(const float *__restrict__ ctrl, const float *__restrict__ eps, int K, int N,
                                int M, float radius, float4 *__restrict__ spheres) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)K * (N + 1)) return;
    const int k = (int)(t / (N + 1)), j = (int)(t % (N + 1));
    const int P = (N + 1) * M + 1;
    // padded control points j .. j + 3 -> control index clamp(j + i - 2, 0, N - 1)
    float q[4][3];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = min(max(j + i - 2, 0), N - 1);
        const bool end = n == 0 || n == N - 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float e = end ? 0.f : eps[((size_t)k * N + n) * 3 + a];
            q[i][a] = __fadd_rn(ctrl[3 * n + a], e);
        }
    }
    float4 *out = spheres + (size_t)k * P + (size_t)j * M;
    for (int m = 0; m < M; ++m) {
        const float u = __fdiv_rn((float)m, (float)M);
        const float u2 = __fmul_rn(u, u), u3 = __fmul_rn(u2, u), v = __fsub_rn(1.f, u);
        const float b0 = __fdiv_rn(__fmul_rn(__fmul_rn(v, v), v), 6.f);
        const float b1 = __fdiv_rn(__fadd_rn(__fsub_rn(__fmul_rn(3.f, u3), __fmul_rn(6.f, u2)), 4.f), 6.f);
        const float b2 = __fdiv_rn(
            __fadd_rn(__fadd_rn(__fsub_rn(__fmul_rn(3.f, u2), __fmul_rn(3.f, u3)), __fmul_rn(3.f, u)), 1.f), 6.f);
        const float b3 = __fdiv_rn(u3, 6.f);
        float x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            x[a] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(b0, q[0][a]), __fmul_rn(b1, q[1][a])), __fmul_rn(b2, q[2][a])),
                             __fmul_rn(b3, q[3][a]));
        out[m] = make_float4(x[0], x[1], x[2], radius);
    }
    if (j == N) spheres[(size_t)k * P + P - 1] = make_float4(ctrl[3 * (N - 1)], ctrl[3 * (N - 1) + 1],
                                                             ctrl[3 * (N - 1) + 2], radius);
}

// One thread per rollout: w_length times the polyline length, in point order.
__global__ void k_refine_length(const float4 *__restrict__ spheres, int K, int P, float w_length,
                                float *__restrict__ tc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const float4 *p = spheres + (size_t)k * P;
    float L = 0.f;
    float4 a = p[0];
    for (int i = 1; i < P; ++i) {
        const float4 b = p[i];
        const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
        L += sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        a = b;
    }
    tc[k] = w_length * L;
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
    c.fixed_ends = 0;
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
    q.sweep_count = 0;
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
    NvtxRange range("cs.mppi_step");
    return mppi_common(scene, desc, x0, U, eps, U_out, cost, weights, collide, params, nullptr);
}

}  // extern "C"

extern "C" {

cs_status cs_path_refine(const cs_scene *scene, const cs_refine_desc *d, const float *ctrl, const float *eps,
                         float *ctrl_out, float *cost, float *weights, const cs_params *params) {
    NvtxRange range("cs.path_refine");
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!d) return invalid("desc is NULL");
    if (d->K < 1 || d->K > (1 << 20)) return invalid("K must lie in [1, 2^20]");
    if (d->N < 2 || d->N > 4096) return invalid("N must lie in [2, 4096]");
    if (d->M < 1 || d->M > 256) return invalid("M must lie in [1, 256]");
    const int64_t P = (int64_t)(d->N + 1) * d->M + 1;
    if ((int64_t)d->K * P > ((int64_t)1 << 26)) return invalid("K * ((N + 1) M + 1) must not exceed 2^26");
    if (!(d->radius > 0.f) || !isfinite(d->radius)) return invalid("radius must be finite and > 0");
    if (!(d->nsigma >= 0.f) || !isfinite(d->nsigma)) return invalid("nsigma must be finite and >= 0");
    if (!(d->lambda > 0.f) || !isfinite(d->lambda)) return invalid("lambda must be finite and > 0");
    if (!(d->w_length >= 0.f) || !isfinite(d->w_length) || !(d->w_collision >= 0.f) || !isfinite(d->w_collision))
        return invalid("cost weights must be finite and >= 0");
    if (!ctrl || !eps || !ctrl_out) return invalid("ctrl, eps and ctrl_out are required");
    if (ctrl_out == ctrl || ctrl_out == eps) return invalid("ctrl_out may not alias ctrl or eps");
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("cs_path_refine takes device buffers only (host_io must be 0)");
    if ((st = check_params(p)) != CS_OK) return st;
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    cudaStream_t s = (cudaStream_t)p.stream;
    const int64_t Q = (int64_t)d->K * P;

    // scratch as for an MPPI iteration of K rollouts x P points
    Workspace *w = nullptr;
    if ((st = get_workspace(sc->device, s, (size_t)Q, false, &w)) != CS_OK) return st;
    if ((st = mppi_reserve(w, d->K, P)) != CS_OK) return st;
    float4 *spheres = reinterpret_cast<float4 *>(w->mppi);
    float *col = w->mppi + 4 * Q, *tc = col + d->K;
    float *c_out = cost ? cost : tc + d->K, *w_out = weights ? weights : c_out + d->K;

    MppiConsts c;
    memset(&c, 0, sizeof(c));
    c.K = d->K;
    c.T = d->N;
    c.radius = d->radius;
    c.w_collision = d->w_collision;
    c.lambda = d->lambda;
    c.fixed_ends = 1;
    const int64_t nthr = (int64_t)d->K * (d->N + 1);
    k_refine_points<<<(unsigned)((nthr + 127) / 128), 128, 0, s>>>(ctrl, eps, d->K, d->N, d->M, d->radius,
                                                                   spheres);
    k_refine_length<<<(d->K + 127) / 128, 128, 0, s>>>(spheres, d->K, (int)P, d->w_length, tc);
    count_launches(2);
    CS_CUDA(cudaGetLastError());
    // the metric of every sample, mean cost per sample summed over the path
    cs_params q = p;
    q.mode = CS_METRIC_MEAN_COST;
    q.group_size = (int32_t)P;
    q.sweep_count = 0;
    q.nsigma_per_query = nullptr;
    q.out_count = nullptr;
    q.out_group_metric = col;
    q.out_group_collide = nullptr;
    q.host_io = 0;
    if ((st = query_common(scene, CS_PRIM_SPHERE, reinterpret_cast<const float *>(spheres), Q, d->nsigma, &q, false,
                           nullptr, nullptr, nullptr, nullptr, w)) != CS_OK)
        return st;
    k_mppi_weights<<<1, kWeightThreads, 0, s>>>(col, tc, c, c_out, w_out);
    k_mppi_update<<<(c.T * 3 * 32 + 255) / 256, 256, 0, s>>>(ctrl, eps, w_out, c, ctrl_out);
    count_launches(2);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // extern "C"
