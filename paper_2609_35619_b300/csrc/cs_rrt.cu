// cs_rrt.cu -- one batched RRT extension with the collision rule of Section
// II-E, the tree resident on the device: for B samples at once, the nearest
// tree node, the steered new node, the collision check of the M points of
// each edge (the query path in flags mode: a point stops once its flag is
// settled, an edge once one of its points collides), and the insertion of
// the free edges' new nodes in sample order.
//
// Nearest node, steering and edge points are computed with correctly rounded
// FP32 operations in a fixed order (no contraction into fused multiply-adds),
// so they are reproducible exactly; ties in the nearest node go to the lowest
// index.
#include <cuda_runtime.h>

#include <math.h>

#include "cs_internal.cuh"

namespace cs {

namespace {

struct RrtConsts {
    int B, M, capacity;
    float step, radius;
};

// One warp per sample: nearest of nodes[0, count) (lane-strided, then a
// fixed tree preferring the smaller index on equal distances), then the new
// node and the M edge points (as float4 spheres of the robot radius).
__global__ void k_rrt_nearest_steer(const float *__restrict__ nodes, const int32_t *__restrict__ count,
                                    const float *__restrict__ samples, RrtConsts c, int32_t *__restrict__ near,
                                    float4 *__restrict__ newn, float4 *__restrict__ pts) {
    const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= c.B) return;  // whole warps leave together
    const int n = min(*count, c.capacity);
    const float sx = samples[3 * b], sy = samples[3 * b + 1], sz = samples[3 * b + 2];
    float best = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
        const float dx = __fsub_rn(nodes[3 * i], sx), dy = __fsub_rn(nodes[3 * i + 1], sy),
                    dz = __fsub_rn(nodes[3 * i + 2], sz);
        const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        if (d2 < best) {  // increasing i per lane: the first minimum stays
            best = d2;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    if (n < 1) bi = -1;  // an empty tree has no node to extend
    const float xn = bi >= 0 ? nodes[3 * bi] : sx, yn = bi >= 0 ? nodes[3 * bi + 1] : sy,
                zn = bi >= 0 ? nodes[3 * bi + 2] : sz;
    // steer: the sample within reach, else step along the direction
    const float dx = __fsub_rn(sx, xn), dy = __fsub_rn(sy, yn), dz = __fsub_rn(sz, zn);
    const float L = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz)));
    float nx = sx, ny = sy, nz = sz;
    if (!(L <= c.step)) {
        const float f = __fdiv_rn(c.step, L);
        nx = __fadd_rn(xn, __fmul_rn(dx, f));
        ny = __fadd_rn(yn, __fmul_rn(dy, f));
        nz = __fadd_rn(zn, __fmul_rn(dz, f));
    }
    if (lane == 0) {
        near[b] = bi;
        newn[b] = make_float4(nx, ny, nz, 0.f);
    }
    const float ex = __fsub_rn(nx, xn), ey = __fsub_rn(ny, yn), ez = __fsub_rn(nz, zn);
    for (int m = lane; m < c.M; m += 32) {
        float4 p = make_float4(nx, ny, nz, c.radius);
        if (m < c.M - 1) {
            const float t = __fdiv_rn((float)(m + 1), (float)c.M);
            p.x = __fadd_rn(xn, __fmul_rn(ex, t));
            p.y = __fadd_rn(yn, __fmul_rn(ey, t));
            p.z = __fadd_rn(zn, __fmul_rn(ez, t));
        }
        pts[(size_t)b * c.M + m] = p;
    }
}

// One block: the free edges' new nodes appended in sample order while the
// capacity lasts; the node count advanced once.
__global__ void __launch_bounds__(1024) k_rrt_insert(float *__restrict__ nodes, int32_t *__restrict__ parent,
                                                     int32_t *__restrict__ count, const int32_t *__restrict__ near,
                                                     const float4 *__restrict__ newn,
                                                     const uint8_t *__restrict__ edge_collide, RrtConsts c,
                                                     int32_t *__restrict__ near_out, uint8_t *__restrict__ free_out) {
    __shared__ int warp_free[32];
    __shared__ int base;
    const int b = threadIdx.x, lane = b & 31, w = b >> 5;
    if (b == 0) base = *count;
    const bool fr = b < c.B && near[b] >= 0 && edge_collide[b] == 0;
    const unsigned m = __ballot_sync(0xffffffffu, fr);
    if (lane == 0) warp_free[w] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_free[k];
    const int rank = before + __popc(m & ((1u << lane) - 1u));
    const int idx = base + rank;
    if (b < c.B) {
        if (near_out) near_out[b] = near[b];
        if (free_out) free_out[b] = fr ? 1 : 0;
    }
    if (fr && idx < c.capacity) {
        const float4 p = newn[b];
        nodes[3 * (size_t)idx] = p.x;
        nodes[3 * (size_t)idx + 1] = p.y;
        nodes[3 * (size_t)idx + 2] = p.z;
        parent[idx] = near[b];
    }
    __syncthreads();
    if (b == 0) {
        int total = 0;
        for (int k = 0; k < 32; ++k) total += warp_free[k];
        *count = min(c.capacity, base + total);
    }
}

}  // namespace

// Scratch of an extension of B samples x M edge points, grown before use so
// that a captured extension allocates nothing: edge points [B M, 4], new
// nodes [B, 4], nearest [B], edge flags [B].
cs_status rrt_reserve(Workspace *w, int B, int M) {
    const int64_t Q = (int64_t)B * M;
    cs_status st = grow_workspace(w, (size_t)Q, false);
    if (st != CS_OK) return st;
    const size_t need = 4 * (size_t)Q + 4 * (size_t)B + (size_t)B + ((size_t)B + 3) / 4;
    if (w->cap_rrt < need) {
        if (w->rrt) CS_CUDA(cudaFree(w->rrt));
        w->rrt = nullptr;
        w->cap_rrt = 0;
        CS_CUDA(cudaMalloc(&w->rrt, 4 * need));
        w->cap_rrt = need;
    }
    return CS_OK;
}

cs_status rrt_check(const cs_scene *scene, const cs_rrt_desc *d, const float *nodes, const int32_t *parent,
                    const int32_t *count, const float *samples) {
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!d) return invalid("desc is NULL");
    if (d->B < 1 || d->B > 1024) return invalid("B must lie in [1, 1024]");
    if (d->M < 2 || d->M > 1024) return invalid("M must lie in [2, 1024]");
    if ((int64_t)d->B * d->M > ((int64_t)1 << 20)) return invalid("B * M must not exceed 2^20");
    if (!(d->step > 0.f) || !isfinite(d->step)) return invalid("step must be finite and > 0");
    if (!(d->radius > 0.f) || !isfinite(d->radius)) return invalid("radius must be finite and > 0");
    if (!(d->nsigma >= 0.f) || !isfinite(d->nsigma)) return invalid("nsigma must be finite and >= 0");
    if (d->capacity < 1) return invalid("capacity must be >= 1");
    if (!nodes || !parent || !count || !samples) return invalid("nodes, parent, count and samples are required");
    return CS_OK;
}

cs_status rrt_common(const cs_scene *scene, const cs_rrt_desc *d, float *nodes, int32_t *parent, int32_t *count,
                     const float *samples, int32_t *nearest, uint8_t *edge_free, const cs_params *params,
                     Workspace *own_ws) {
    cs_status st = rrt_check(scene, d, nodes, parent, count, samples);
    if (st != CS_OK) return st;
    cs_params p;
    if (params) p = *params;
    else cs_params_init(&p);
    if (p.host_io) return invalid("cs_rrt_extend takes device buffers only (host_io must be 0)");
    if ((st = check_params(p)) != CS_OK) return st;
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    cudaStream_t s = (cudaStream_t)p.stream;
    const int64_t Q = (int64_t)d->B * d->M;

    Workspace *w = own_ws;
    if (!w && (st = get_workspace(sc->device, s, (size_t)Q, false, &w)) != CS_OK) return st;
    if ((st = rrt_reserve(w, d->B, d->M)) != CS_OK) return st;
    float4 *pts = reinterpret_cast<float4 *>(w->rrt);
    float4 *newn = pts + Q;
    int32_t *near = reinterpret_cast<int32_t *>(newn + d->B);
    uint8_t *gcol = reinterpret_cast<uint8_t *>(near + d->B);

    RrtConsts c;
    c.B = d->B;
    c.M = d->M;
    c.capacity = d->capacity;
    c.step = d->step;
    c.radius = d->radius;
    k_rrt_nearest_steer<<<(unsigned)((c.B * 32 + 255) / 256), 256, 0, s>>>(nodes, count, samples, c, near, newn,
                                                                          pts);
    count_launches(1);
    CS_CUDA(cudaGetLastError());
    // the edges' points in flags mode: an edge stops at its first colliding point
    cs_params q = p;
    q.mode = CS_METRIC_FLAGS;
    q.group_size = d->M;
    q.sweep_count = 0;
    q.nsigma_per_query = nullptr;
    q.out_count = nullptr;
    q.out_group_metric = nullptr;
    q.out_group_collide = gcol;
    q.host_io = 0;
    if ((st = query_common(scene, CS_PRIM_SPHERE, reinterpret_cast<const float *>(pts), Q, d->nsigma, &q, false,
                           nullptr, nullptr, nullptr, nullptr, w)) != CS_OK)
        return st;
    k_rrt_insert<<<1, 1024, 0, s>>>(nodes, parent, count, near, newn, gcol, c, nearest, edge_free);
    count_launches(1);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_rrt_extend(const cs_scene *scene, const cs_rrt_desc *d, float *nodes, int32_t *parent,
                        int32_t *count, const float *samples, int32_t *nearest, uint8_t *edge_free,
                        const cs_params *params) {
    NvtxRange range("cs.rrt_extend");
    return rrt_common(scene, d, nodes, parent, count, samples, nearest, edge_free, params, nullptr);
}

}  // extern "C"
