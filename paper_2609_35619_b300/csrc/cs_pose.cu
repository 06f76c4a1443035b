// cs_pose.cu -- the pose chain that turns per-waypoint rigid poses into the
// sphere centres the metric consumes, and its adjoint.  A pose is (t, w):
// translation t and axis-angle rotation w, R(w) = exp([w]x) (Rodrigues);
// sphere k of a pose sits at t + R(w) p_k.
#include <math.h>

#include "cs_internal.cuh"

namespace cs {

namespace {

// Coefficients of R = I + a [w]x + b [w]x^2 and of the left Jacobian
// J_l = I + b [w]x + c [w]x^2: a = sin(t)/t, b = (1 - cos t)/t^2 written as
// 2 sin^2(t/2)/t^2 (no cancellation), c = (t - sin t)/t^3 from its Taylor
// series below 0.5 rad.
__device__ __forceinline__ void rod_coeffs(float th, float &a, float &b, float &c) {
    float t2 = th * th;
    if (th < 1e-3f) {
        a = 1.f - t2 * (1.f / 6.f);
        b = 0.5f - t2 * (1.f / 24.f);
    } else {
        float s, co;
        sincosf(th, &s, &co);
        float sh = sinf(0.5f * th);
        a = s / th;
        b = 2.f * sh * sh / t2;
    }
    if (th < 0.5f) {
        c = (1.f / 6.f) - t2 * ((1.f / 120.f) - t2 * ((1.f / 5040.f) - t2 * (1.f / 362880.f)));
    } else {
        c = (th - sinf(th)) / (t2 * th);
    }
}

struct Rot3 {
    float m[3][3];
};

__device__ __forceinline__ Rot3 rodrigues(float wx, float wy, float wz, float a, float b) {
    // R = I + a K + b K^2, K = [w]x, K^2 = w w^T - |w|^2 I
    float n2 = wx * wx + wy * wy + wz * wz;
    Rot3 R;
    R.m[0][0] = 1.f + b * (wx * wx - n2);
    R.m[1][1] = 1.f + b * (wy * wy - n2);
    R.m[2][2] = 1.f + b * (wz * wz - n2);
    R.m[0][1] = -a * wz + b * wx * wy;
    R.m[1][0] = a * wz + b * wx * wy;
    R.m[0][2] = a * wy + b * wx * wz;
    R.m[2][0] = -a * wy + b * wx * wz;
    R.m[1][2] = -a * wx + b * wy * wz;
    R.m[2][1] = a * wx + b * wy * wz;
    return R;
}

__global__ void k_pose_spheres(const float *__restrict__ poses, int64_t P,
                               const float *__restrict__ offsets, int K, float radius,
                               float *__restrict__ out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * K) return;
    int64_t p = idx / K;
    int k = (int)(idx - p * K);
    const float *ps = poses + 6 * p;
    float wx = ps[3], wy = ps[4], wz = ps[5];
    float th = sqrtf(wx * wx + wy * wy + wz * wz);
    float a, b, c;
    rod_coeffs(th, a, b, c);
    Rot3 R = rodrigues(wx, wy, wz, a, b);
    float ox = offsets[3 * k], oy = offsets[3 * k + 1], oz = offsets[3 * k + 2];
    float4 r;
    r.x = ps[0] + R.m[0][0] * ox + R.m[0][1] * oy + R.m[0][2] * oz;
    r.y = ps[1] + R.m[1][0] * ox + R.m[1][1] * oy + R.m[1][2] * oz;
    r.z = ps[2] + R.m[2][0] * ox + R.m[2][1] * oy + R.m[2][2] * oz;
    r.w = radius;
    float *o = out + 4 * idx;
    o[0] = r.x; o[1] = r.y; o[2] = r.z; o[3] = r.w;
}

// grad_t = sum_k g_k;  grad_w = J_l(w)^T sum_k (R p_k) x g_k.
__global__ void k_pose_grad(const float *__restrict__ poses, int64_t P,
                            const float *__restrict__ offsets, int K,
                            const float *__restrict__ gc, float *__restrict__ gp) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const float *ps = poses + 6 * p;
    float wx = ps[3], wy = ps[4], wz = ps[5];
    float th = sqrtf(wx * wx + wy * wy + wz * wz);
    float a, b, c;
    rod_coeffs(th, a, b, c);
    Rot3 R = rodrigues(wx, wy, wz, a, b);
    float gt[3] = {0, 0, 0}, tq[3] = {0, 0, 0};
    for (int k = 0; k < K; ++k) {
        const float *g = gc + 3 * (p * K + k);
        float ox = offsets[3 * k], oy = offsets[3 * k + 1], oz = offsets[3 * k + 2];
        float rx = R.m[0][0] * ox + R.m[0][1] * oy + R.m[0][2] * oz;
        float ry = R.m[1][0] * ox + R.m[1][1] * oy + R.m[1][2] * oz;
        float rz = R.m[2][0] * ox + R.m[2][1] * oy + R.m[2][2] * oz;
        gt[0] += g[0]; gt[1] += g[1]; gt[2] += g[2];
        tq[0] += ry * g[2] - rz * g[1];
        tq[1] += rz * g[0] - rx * g[2];
        tq[2] += rx * g[1] - ry * g[0];
    }
    // J_l = I + b K + c K^2 (K = [w]x); J_l^T v = v - b (w x v) + c K^2 v
    float n2 = wx * wx + wy * wy + wz * wz;
    float wv = wx * tq[0] + wy * tq[1] + wz * tq[2];
    float cx_ = wy * tq[2] - wz * tq[1], cy_ = wz * tq[0] - wx * tq[2], cz_ = wx * tq[1] - wy * tq[0];
    float *o = gp + 6 * p;
    o[0] = gt[0]; o[1] = gt[1]; o[2] = gt[2];
    o[3] = tq[0] - b * cx_ + c * (wx * wv - n2 * tq[0]);
    o[4] = tq[1] - b * cy_ + c * (wy * wv - n2 * tq[1]);
    o[5] = tq[2] - b * cz_ + c * (wz * wv - n2 * tq[2]);
}

}  // namespace

void launch_pose(const float *poses, int64_t P, const float *offsets, int K, float radius,
                 float *out, cudaStream_t s) {
    int64_t n = P * K;
    k_pose_spheres<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(poses, P, offsets, K, radius, out);
    count_launches(1);
}

void launch_pose_grad(const float *poses, int64_t P, const float *offsets, int K, const float *gc,
                      float *gp, cudaStream_t s) {
    k_pose_grad<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(poses, P, offsets, K, gc, gp);
    count_launches(1);
}

}  // namespace cs
