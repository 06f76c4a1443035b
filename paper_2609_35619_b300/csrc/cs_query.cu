// cs_query.cu -- the query path: spatial ordering of the primitives, the
// fused cull + pair evaluation + per-primitive reduction kernel (forward and
// adjoint), and the group epilogue.
//
// Fused kernel layout (one CTA per tile of TQ consecutive sorted primitives):
//   warps 0..NCW-1  consumers: each lane holds QB primitives in registers and
//                   streams the staged Gaussians from shared memory, updating
//                   its per-primitive reductions (no cross-lane traffic);
//   warp NCW        producer: computes the tile's bounding box and reach,
//                   walks the grid rows it can reach (the cull) and the
//                   large-tier chunks, and stages the reachable Gaussian
//                   spans into a ring of NS shared-memory stages with 1-D bulk
//                   copies completing on per-stage mbarriers.
// Before evaluating a staged chunk of 32 Gaussians each consumer warp tests
// the chunk's bounding record against its own primitives (warp-level cull).
#include <math.h>

#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

// ----------------------------------------------------------- parameters
struct QueryConsts {
    float S_cut;    // neighbour cutoff s_min + ln(1/eps)/gamma
    float S_reach;  // max(S_cut, 1): the cull keeps every pair below it
    float T_in;     // st2 < T_in  <=>  st2 < 1 and st2 <= S_cut
    float G;        // gamma * log2(e)
    float Gsmin;    // G * s_min
    float s_min;
    float d_max;
    float gamma;
    float tau;
    float K;        // 1 / (tau ln 2): softmin in base 2
    int k_thr;
    int mode;
    int group_size;
};

struct EvalArgs {
    SceneDev sc;
    const float4 *qrec;      // prepared primitives, sorted order, RECS float4 each
    const float *qns;        // n_sigma per sorted primitive
    const uint32_t *perm;    // sorted position -> input row
    int Q;
    QueryConsts k;
    float *out_metric;
    uint8_t *out_collide;
    int32_t *out_count;
    const float *grad_out;   // GRAD: upstream per row (or per group)
    float *grad_centres;     // GRAD: [Q,3]
    unsigned *err;
    unsigned long long *stats;
    long long wait_polls;
};

constexpr int kNS = 4;      // pipeline stages
constexpr int kCH = 128;    // Gaussians per stage
constexpr int kMaxP = 32;   // pieces (contiguous spans) per stage

struct StageMeta {
    int count;
    int npieces;
    int pad[2];
    int4 piece[kMaxP];  // (offset in stage, first sorted index, count, 0)
};

struct __align__(16) EvalSmem {
    float4 pos[kNS][kCH];
    float4 covA[kNS][kCH];
    float4 covB[kNS][kCH];
    StageMeta meta[kNS];
    uint64_t full[kNS];
    uint64_t empty[kNS];
    int abort;  // an earlier launch on this stream timed out: skip the work
};

template <int PRIM> struct PrimTraits;
template <> struct PrimTraits<0> { static constexpr int RECS = 1; };  // sphere: (c, r)
template <> struct PrimTraits<1> { static constexpr int RECS = 3; };  // ellipsoid

// Cull parameters of one prepared primitive: every pair farther than
// alpha*s + sqrt(alpha^2 s^2 + beta) (s = the Gaussian's largest scale) has
// st2 > S_reach.  Sphere: alpha = n, beta = S r^2.  Ellipsoid (semi-axes
// a_max >= ... >= a_min): alpha = n a_max^2/a_min^2, beta = S a_max^2.
template <int PRIM>
__device__ __forceinline__ void prim_reach(const float4 *rec, float ns, float S, float &alpha,
                                           float &beta) {
    if (PRIM == 0) {
        float r = rec[0].w;
        alpha = ns;
        beta = S * r * r;
    } else {
        float amax = rec[0].w, amin = rec[2].z;
        alpha = ns * (amax * amax) / (amin * amin);
        beta = S * amax * amax;
    }
}

__device__ __forceinline__ bool rec_valid(const float4 &r0) { return !isnan(r0.w); }

__device__ __forceinline__ float box_gap2(float lx, float ly, float lz, float hx, float hy, float hz,
                                          float4 blo, float4 bhi) {
    float gx = fmaxf(0.f, fmaxf(blo.x - hx, lx - bhi.x));
    float gy = fmaxf(0.f, fmaxf(blo.y - hy, ly - bhi.y));
    float gz = fmaxf(0.f, fmaxf(blo.z - hz, lz - bhi.z));
    return fmaf(gx, gx, fmaf(gy, gy, gz * gz));
}

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait by poll count and wall time (1 s; a healthy wait is a few
// microseconds).
__device__ __noinline__ bool wait_phase(uint64_t *bar, unsigned parity, long long polls) {
    long long t0 = globaltimer_ns();
    for (long long i = 0; i < polls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && globaltimer_ns() - t0 > 1000000000ll) break;
    }
    return false;
}

__device__ __forceinline__ int cell_of(float x, float lo, float inv_h, int dim) {
    int c = (int)floorf((x - lo) * inv_h);
    return min(max(c, 0), dim - 1);
}

// ------------------------------------------------------------- producer
struct Producer {
    EvalSmem *sm;
    const SceneDev *sc;
    long long polls;
    int k = 0;       // stage sequence number
    int fill = 0;    // Gaussians in the open stage
    int np = 0;      // pieces in the open stage
    bool failed = false;
    int lane;

    __device__ void open_stage() {
        int s = k % kNS;
        if (k >= kNS) {
            bool ok = true;
            if (lane == 0) ok = wait_phase(&sm->empty[s], (unsigned)((k / kNS - 1) & 1), polls);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) failed = true;
        }
        fill = 0;
        np = 0;
    }
    __device__ void close_stage() {
        int s = k % kNS;
        if (lane == 0) {
            sm->meta[s].count = fill;
            sm->meta[s].npieces = np;
            mbar_arrive(&sm->full[s]);
        }
        __syncwarp();
        ++k;
        open_stage();
    }
    // Append sorted Gaussians [start, start + cnt) to the staged stream.
    __device__ void append(int start, int cnt) {
        while (cnt > 0 && !failed) {
            int s = k % kNS;
            int take = min(cnt, kCH - fill);
            if (lane == 0) {
                sm->meta[s].piece[np] = make_int4(fill, start, take, 0);
                unsigned bytes = (unsigned)take * 16u;
                mbar_expect_tx(&sm->full[s], 3u * bytes);
                bulk_g2s(&sm->pos[s][fill], sc->pos + start, bytes, &sm->full[s]);
                bulk_g2s(&sm->covA[s][fill], sc->covA + start, bytes, &sm->full[s]);
                bulk_g2s(&sm->covB[s][fill], sc->covB + start, bytes, &sm->full[s]);
            }
            fill += take;
            start += take;
            cnt -= take;
            ++np;
            if (fill == kCH || np == kMaxP) close_stage();
        }
    }
    __device__ void finish() {
        if (failed) return;
        if (fill > 0) close_stage();
        if (failed) return;
        int s = k % kNS;
        if (lane == 0) {
            sm->meta[s].count = 0;  // terminator
            sm->meta[s].npieces = 0;
            mbar_arrive(&sm->full[s]);
        }
        __syncwarp();
    }
    // After a failed wait: close the open stage so its copies can complete,
    // then wait (bounded) for every stage's latest phase.
    __device__ void drain() {
        if (lane == 0) {
            int s = k % kNS;
            if (fill > 0) {
                sm->meta[s].count = fill;
                sm->meta[s].npieces = np;
                mbar_arrive(&sm->full[s]);
                ++k;
            }
            for (int j = max(0, k - kNS); j < k; ++j)
                wait_phase(&sm->full[j % kNS], (unsigned)((j / kNS) & 1), polls);
        }
        __syncwarp();
    }
};

template <int PRIM, int QB, int NCW>
__device__ void producer_warp(const EvalArgs &a, EvalSmem *sm, int tile) {
    constexpr int RECS = PrimTraits<PRIM>::RECS;
    constexpr int TQ = NCW * 32 * QB;
    const int lane = threadIdx.x & 31;
    const SceneDev &sc = a.sc;
    // tile bounding box and reach parameters over its valid primitives
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY,
          hz = -INFINITY, al = 0.f, be = 0.f;
    const int q0 = tile * TQ;
    for (int t = lane; t < TQ; t += 32) {
        int q = q0 + t;
        if (q >= a.Q) break;
        const float4 *rec = a.qrec + (size_t)q * RECS;
        float4 r0 = rec[0];
        if (!rec_valid(r0)) continue;
        float alpha, beta;
        prim_reach<PRIM>(rec, a.qns[q], a.k.S_reach, alpha, beta);
        lx = fminf(lx, r0.x); ly = fminf(ly, r0.y); lz = fminf(lz, r0.z);
        hx = fmaxf(hx, r0.x); hy = fmaxf(hy, r0.y); hz = fmaxf(hz, r0.z);
        al = fmaxf(al, alpha);
        be = fmaxf(be, beta);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        al = fmaxf(al, __shfl_xor_sync(0xffffffffu, al, o));
        be = fmaxf(be, __shfl_xor_sync(0xffffffffu, be, o));
    }
    Producer pr{sm, &sc, a.wait_polls};
    pr.lane = lane;
    const bool any = lx <= hx;  // at least one valid primitive
    if (any && sc.n_grid > 0) {
        // ---- grid rows within reach of the tile box (sigma = grid-tier max)
        const float R = reach(al, be, sc.sigma_tier, sc.pad_abs);
        const float R2 = R * R;
        const int iy0 = cell_of(ly - R, sc.lo[1], sc.inv_h, sc.dims[1]);
        const int iy1 = cell_of(hy + R, sc.lo[1], sc.inv_h, sc.dims[1]);
        const int iz0 = cell_of(lz - R, sc.lo[2], sc.inv_h, sc.dims[2]);
        const int iz1 = cell_of(hz + R, sc.lo[2], sc.inv_h, sc.dims[2]);
        const int ny = iy1 - iy0 + 1;
        const int nrows = ny * (iz1 - iz0 + 1);
        const float slack = sc.pad_abs;
        for (int rb = 0; rb < nrows && !pr.failed; rb += 32) {
            int r = rb + lane;
            int start = 0, cnt = 0;
            if (r < nrows) {
                int iz = iz0 + r / ny, iy = iy0 + r % ny;
                float y0 = sc.lo[1] + (float)iy * sc.h - slack, y1 = sc.lo[1] + (float)(iy + 1) * sc.h + slack;
                float z0 = sc.lo[2] + (float)iz * sc.h - slack, z1 = sc.lo[2] + (float)(iz + 1) * sc.h + slack;
                // first and last rows extend to infinity (clamped cell coordinates)
                if (iy == 0) y0 = -INFINITY;
                if (iy == sc.dims[1] - 1) y1 = INFINITY;
                if (iz == 0) z0 = -INFINITY;
                if (iz == sc.dims[2] - 1) z1 = INFINITY;
                float gy = fmaxf(0.f, fmaxf(y0 - hy, ly - y1));
                float gz = fmaxf(0.f, fmaxf(z0 - hz, lz - z1));
                float d2 = fmaf(gy, gy, gz * gz);
                if (d2 <= R2) {
                    float half = sqrtf(R2 - d2);
                    int ix0 = cell_of(lx - half, sc.lo[0], sc.inv_h, sc.dims[0]);
                    int ix1 = cell_of(hx + half, sc.lo[0], sc.inv_h, sc.dims[0]);
                    uint32_t rowkey = (uint32_t)sc.dims[0] * ((uint32_t)iy + (uint32_t)sc.dims[1] * (uint32_t)iz);
                    uint32_t b = sc.cell_start[rowkey + ix0];
                    uint32_t e = sc.cell_start[rowkey + ix1 + 1];
                    start = (int)b;
                    cnt = (int)(e - b);
                }
            }
            unsigned m = __ballot_sync(0xffffffffu, cnt > 0);
            while (m) {
                int src = __ffs(m) - 1;
                m &= m - 1;
                int s0 = __shfl_sync(0xffffffffu, start, src);
                int c0 = __shfl_sync(0xffffffffu, cnt, src);
                pr.append(s0, c0);
                if (pr.failed) break;
            }
        }
    }
    if (any && sc.n_kept > sc.n_grid && !pr.failed) {
        // ---- large tier: chunk records tested one by one against the tile box
        const int c_begin = sc.n_grid / kChunk;
        for (int cb = c_begin; cb < sc.nchunks && !pr.failed; cb += 32) {
            int c = cb + lane;
            bool pass = false;
            if (c < sc.nchunks) {
                float4 clo = sc.chunk_lo[c], chi = sc.chunk_hi[c];
                float Rc = reach(al, be, clo.w, sc.pad_abs);
                pass = box_gap2(lx, ly, lz, hx, hy, hz, clo, chi) <= Rc * Rc;
            }
            unsigned m = __ballot_sync(0xffffffffu, pass);
            while (m) {
                int src = __ffs(m) - 1;
                m &= m - 1;
                int cc = cb + src;
                int s0 = max(cc * kChunk, sc.n_grid);
                int e0 = min(cc * kChunk + kChunk, sc.n_kept);
                pr.append(s0, e0 - s0);
                if (pr.failed) break;
            }
        }
    }
    pr.finish();
    if (pr.failed) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        pr.drain();
    }
}

// ------------------------------------------------------------- consumers
template <int PRIM, int QB, bool SOFTMIN, bool GRAD>
struct Lane;

// Per-lane state for QB spheres.
template <int QB, bool SOFTMIN, bool GRAD>
struct Lane<0, QB, SOFTMIN, GRAD> {
    float cx[QB], cy[QB], cz[QB], ir2[QB], ns2[QB];
    float sum[QB], cnt[QB], cin[QB], mn[QB];
    float sm_m[QB], sm_acc[QB];
    float gx[QB], gy[QB], gz[QB];

    __device__ void init(const float4 *rec, const float *ns, int i) {
        float4 r = rec[0];
        cx[i] = r.x; cy[i] = r.y; cz[i] = r.z;
        ir2[i] = 1.f / (r.w * r.w);
        ns2[i] = 2.f * ns[0];
    }
    __device__ void clear(int i) {
        sum[i] = 0.f; cnt[i] = 0.f; cin[i] = 0.f; mn[i] = INFINITY;
        sm_m[i] = INFINITY; sm_acc[i] = 0.f;
        gx[i] = gy[i] = gz[i] = 0.f;
    }
    // a slot without a valid primitive: finite values, results never stored
    __device__ void park(int i) { cx[i] = cy[i] = cz[i] = 0.f; ir2[i] = 0.f; ns2[i] = 0.f; }
    // Eq. 5, 7, 8, 11 for one Gaussian against the lane's QB spheres.  In the
    // difference form d = mu - c (no cancellation in absolute coordinates):
    //   s^2 = |d|^2 / r^2,  sqrt(sigma^2) = 2 sqrt(d^T Sigma d) / r^2,
    //   st^2 = max(0, |d|^2 - 2 n sqrt(d^T Sigma d)) / r^2.
    __device__ __forceinline__ void update(const float4 P, const float4 A, const float4 B,
                                           const QueryConsts &k) {
#pragma unroll
        for (int i = 0; i < QB; ++i) {
            float dx = P.x - cx[i], dy = P.y - cy[i], dz = P.z - cz[i];
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float q, vx = 0.f, vy = 0.f, vz = 0.f;
            if (!GRAD) {
                float t1 = fmaf(B.x, dz, fmaf(A.w, dy, A.x * dx));  // Sxx dx + 2Sxy dy + 2Sxz dz
                float t2 = fmaf(B.y, dz, A.y * dy);                 // Syy dy + 2Syz dz
                q = fmaf(dx, t1, fmaf(dy, t2, dz * (A.z * dz)));
            } else {
                // Sigma d with the stored doubled off-diagonals halved
                float hxy = 0.5f * A.w, hxz = 0.5f * B.x, hyz = 0.5f * B.y;
                vx = fmaf(hxz, dz, fmaf(hxy, dy, A.x * dx));
                vy = fmaf(hyz, dz, fmaf(A.y, dy, hxy * dx));
                vz = fmaf(A.z, dz, fmaf(hyz, dy, hxz * dx));
                q = fmaf(dx, vx, fmaf(dy, vy, dz * vz));
            }
            q = fmaxf(q, 0.f);
            float sq = sqrt_approx(q);
            float raw = fmaf(-ns2[i], sq, r2);
            float st2 = fmaxf(raw, 0.f) * ir2[i];
            float dc = ex2_approx(fminf(fmaf(st2, -k.G, k.Gsmin), 0.f));
            bool nb = st2 <= k.S_cut;
            if (!GRAD) {
                if (nb) { sum[i] += dc; cnt[i] += 1.f; }
                if (st2 < k.T_in) cin[i] += 1.f;
                mn[i] = fminf(mn[i], st2);
                if (SOFTMIN && nb) {
                    float nm = fminf(sm_m[i], st2);
                    sm_acc[i] = fmaf(sm_acc[i], ex2_approx((nm - sm_m[i]) * k.K),
                                     ex2_approx((nm - st2) * k.K));
                    sm_m[i] = nm;
                }
            } else {
                // d st2 / d c = (-2 d + 2 n Sigma d / sqrt(d^T Sigma d)) / r^2 where raw > 0
                float rs = sq > 0.f ? ns2[i] / sq : 0.f;
                float live = raw > 0.f ? ir2[i] : 0.f;
                float ex = (fmaf(rs, vx, -2.f * dx)) * live;
                float ey = (fmaf(rs, vy, -2.f * dy)) * live;
                float ez = (fmaf(rs, vz, -2.f * dz)) * live;
                if (nb) cnt[i] += 1.f;
                if (k.mode <= CS_METRIC_SUM_COST) {
                    // Eq. 11 is flat below s_min
                    float w = (nb && st2 > k.s_min) ? dc : 0.f;
                    gx[i] = fmaf(w, ex, gx[i]); gy[i] = fmaf(w, ey, gy[i]); gz[i] = fmaf(w, ez, gz[i]);
                } else if (k.mode == CS_METRIC_MIN_S2) {
                    if (nb && st2 < mn[i]) { mn[i] = st2; gx[i] = ex; gy[i] = ey; gz[i] = ez; }
                } else if (nb) {
                    float nm = fminf(sm_m[i], st2);
                    float f = ex2_approx((nm - sm_m[i]) * k.K);
                    float e = ex2_approx((nm - st2) * k.K);
                    sm_acc[i] = fmaf(sm_acc[i], f, e);
                    gx[i] = fmaf(gx[i], f, e * ex); gy[i] = fmaf(gy[i], f, e * ey); gz[i] = fmaf(gz[i], f, e * ez);
                    sm_m[i] = nm;
                }
            }
        }
    }
};

// Per-lane state for QB ellipsoids: centre, A (6 coefficients), 2 n.
template <int QB, bool SOFTMIN, bool GRAD>
struct Lane<1, QB, SOFTMIN, GRAD> {
    float cx[QB], cy[QB], cz[QB], axx[QB], ayy[QB], azz[QB], axy[QB], axz[QB], ayz[QB], ns2[QB];
    float sum[QB], cnt[QB], cin[QB], mn[QB];
    float sm_m[QB], sm_acc[QB];
    float gx[QB], gy[QB], gz[QB];

    __device__ void init(const float4 *rec, const float *ns, int i) {
        float4 r0 = rec[0], r1 = rec[1], r2 = rec[2];
        cx[i] = r0.x; cy[i] = r0.y; cz[i] = r0.z;
        axx[i] = r1.x; ayy[i] = r1.y; azz[i] = r1.z; axy[i] = r1.w;
        axz[i] = r2.x; ayz[i] = r2.y;
        ns2[i] = 2.f * ns[0];
    }
    __device__ void clear(int i) {
        sum[i] = 0.f; cnt[i] = 0.f; cin[i] = 0.f; mn[i] = INFINITY;
        sm_m[i] = INFINITY; sm_acc[i] = 0.f;
        gx[i] = gy[i] = gz[i] = 0.f;
    }
    __device__ void park(int i) {
        cx[i] = cy[i] = cz[i] = 0.f;
        axx[i] = ayy[i] = azz[i] = axy[i] = axz[i] = ayz[i] = 0.f;
        ns2[i] = 0.f;
    }
    // Eq. 5-8 for an ellipsoid: w = A d, s^2 = d^T w, sqrt(sigma^2) = 2 sqrt(w^T Sigma w).
    __device__ __forceinline__ void update(const float4 P, const float4 A, const float4 B,
                                           const QueryConsts &k) {
#pragma unroll
        for (int i = 0; i < QB; ++i) {
            float dx = P.x - cx[i], dy = P.y - cy[i], dz = P.z - cz[i];
            float wx = fmaf(axz[i], dz, fmaf(axy[i], dy, axx[i] * dx));
            float wy = fmaf(ayz[i], dz, fmaf(ayy[i], dy, axy[i] * dx));
            float wz = fmaf(azz[i], dz, fmaf(ayz[i], dy, axz[i] * dx));
            float s2 = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
            float u, vx = 0.f, vy = 0.f, vz = 0.f;
            if (!GRAD) {
                float t1 = fmaf(B.x, wz, fmaf(A.w, wy, A.x * wx));
                float t2 = fmaf(B.y, wz, A.y * wy);
                u = fmaf(wx, t1, fmaf(wy, t2, wz * (A.z * wz)));
            } else {
                float hxy = 0.5f * A.w, hxz = 0.5f * B.x, hyz = 0.5f * B.y;
                vx = fmaf(hxz, wz, fmaf(hxy, wy, A.x * wx));   // Sigma w
                vy = fmaf(hyz, wz, fmaf(A.y, wy, hxy * wx));
                vz = fmaf(A.z, wz, fmaf(hyz, wy, hxz * wx));
                u = fmaf(wx, vx, fmaf(wy, vy, wz * vz));
            }
            u = fmaxf(u, 0.f);
            float sq = sqrt_approx(u);
            float raw = fmaf(-ns2[i], sq, s2);
            float st2 = fmaxf(raw, 0.f);
            float dc = ex2_approx(fminf(fmaf(st2, -k.G, k.Gsmin), 0.f));
            bool nb = st2 <= k.S_cut;
            if (!GRAD) {
                if (nb) { sum[i] += dc; cnt[i] += 1.f; }
                if (st2 < k.T_in) cin[i] += 1.f;
                mn[i] = fminf(mn[i], st2);
                if (SOFTMIN && nb) {
                    float nm = fminf(sm_m[i], st2);
                    sm_acc[i] = fmaf(sm_acc[i], ex2_approx((nm - sm_m[i]) * k.K),
                                     ex2_approx((nm - st2) * k.K));
                    sm_m[i] = nm;
                }
            } else {
                // d st2 / d c = -2 w + 2 n A Sigma w / sqrt(w^T Sigma w) where raw > 0
                float rs = sq > 0.f ? ns2[i] / sq : 0.f;
                float live = raw > 0.f ? 1.f : 0.f;
                float px = fmaf(axz[i], vz, fmaf(axy[i], vy, axx[i] * vx));  // A Sigma w
                float py = fmaf(ayz[i], vz, fmaf(ayy[i], vy, axy[i] * vx));
                float pz = fmaf(azz[i], vz, fmaf(ayz[i], vy, axz[i] * vx));
                float ex = fmaf(rs, px, -2.f * wx) * live;
                float ey = fmaf(rs, py, -2.f * wy) * live;
                float ez = fmaf(rs, pz, -2.f * wz) * live;
                if (nb) cnt[i] += 1.f;
                if (k.mode <= CS_METRIC_SUM_COST) {
                    float w = (nb && st2 > k.s_min) ? dc : 0.f;
                    gx[i] = fmaf(w, ex, gx[i]); gy[i] = fmaf(w, ey, gy[i]); gz[i] = fmaf(w, ez, gz[i]);
                } else if (k.mode == CS_METRIC_MIN_S2) {
                    if (nb && st2 < mn[i]) { mn[i] = st2; gx[i] = ex; gy[i] = ey; gz[i] = ez; }
                } else if (nb) {
                    float nm = fminf(sm_m[i], st2);
                    float f = ex2_approx((nm - sm_m[i]) * k.K);
                    float e = ex2_approx((nm - st2) * k.K);
                    sm_acc[i] = fmaf(sm_acc[i], f, e);
                    gx[i] = fmaf(gx[i], f, e * ex); gy[i] = fmaf(gy[i], f, e * ey); gz[i] = fmaf(gz[i], f, e * ez);
                    sm_m[i] = nm;
                }
            }
        }
    }
};

template <int PRIM, int QB, int NCW, bool SOFTMIN, bool GRAD>
__device__ void consumer_warp(const EvalArgs &a, EvalSmem *sm, int tile, int warp, bool abort) {
    constexpr int RECS = PrimTraits<PRIM>::RECS;
    constexpr int TQ = NCW * 32 * QB;
    const int lane = threadIdx.x & 31;
    const QueryConsts &k = a.k;
    Lane<PRIM, QB, SOFTMIN, GRAD> st;
    int qi[QB];
    bool valid[QB];
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    float al = 0.f, be = 0.f;
    int nvalid = 0;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
        int q = tile * TQ + warp * 32 * QB + i * 32 + lane;
        qi[i] = q;
        valid[i] = false;
        st.clear(i);
        st.park(i);
        if (q < a.Q) {
            const float4 *rec = a.qrec + (size_t)q * RECS;
            float4 r0 = rec[0];
            if (rec_valid(r0)) {
                valid[i] = true;
                st.init(rec, a.qns + q, i);
                float alpha, beta;
                prim_reach<PRIM>(rec, a.qns[q], k.S_reach, alpha, beta);
                lx = fminf(lx, r0.x); ly = fminf(ly, r0.y); lz = fminf(lz, r0.z);
                hx = fmaxf(hx, r0.x); hy = fmaxf(hy, r0.y); hz = fmaxf(hz, r0.z);
                al = fmaxf(al, alpha); be = fmaxf(be, beta);
                ++nvalid;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        al = fmaxf(al, __shfl_xor_sync(0xffffffffu, al, o));
        be = fmaxf(be, __shfl_xor_sync(0xffffffffu, be, o));
        nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    }
    const bool warp_live = nvalid > 0;
    const SceneDev &sc = a.sc;
    long long evaluated = 0;
    bool ok = !abort;
    for (int kk = 0; ok; ++kk) {
        const int s = kk % kNS;
        bool got = true;
        if (lane == 0) got = wait_phase(&sm->full[s], (unsigned)((kk / kNS) & 1), a.wait_polls);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        const int n = sm->meta[s].count;
        if (n == 0) break;
        if (warp_live) {
            const int npc = sm->meta[s].npieces;
            for (int p = 0; p < npc; ++p) {
                const int4 pc = sm->meta[s].piece[p];
                int g = pc.y;
                const int gend = pc.y + pc.z;
                while (g < gend) {
                    const int c = g >> 5;
                    const int ce = min(gend, (c + 1) << 5);
                    const float4 clo = __ldg(sc.chunk_lo + c);
                    const float4 chi = __ldg(sc.chunk_hi + c);
                    const float Rc = reach(al, be, clo.w, sc.pad_abs);
                    if (box_gap2(lx, ly, lz, hx, hy, hz, clo, chi) <= Rc * Rc) {
                        const int o0 = pc.x + (g - pc.y), o1 = pc.x + (ce - pc.y);
                        evaluated += o1 - o0;
#pragma unroll 2
                        for (int o = o0; o < o1; ++o)
                            st.update(sm->pos[s][o], sm->covA[s][o], sm->covB[s][o], k);
                    }
                    g = ce;
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->empty[s]);
    }
    if (!ok && !abort && lane == 0) atomicOr(a.err, kErrTimeout);

    // ---- outputs (input row order)
    float nb_total = 0.f;
#pragma unroll
    for (int i = 0; i < QB; ++i) {
        const int q = qi[i];
        if (q >= a.Q) continue;
        const uint32_t row = a.perm[q];
        if (!GRAD) {
            float metric;
            uint8_t col = 0;
            int cntv = 0;
            if (!valid[i] || !ok) {
                metric = __int_as_float(0x7fc00000);
            } else {
                const float c = st.cnt[i];
                cntv = (int)c;
                nb_total += c;
                col = st.cin[i] > (float)k.k_thr ? 1 : 0;
                switch (k.mode) {
                    case CS_METRIC_MEAN_COST: metric = c > 0.f ? st.sum[i] * k.d_max / c : 0.f; break;
                    case CS_METRIC_SUM_COST: metric = st.sum[i] * k.d_max; break;
                    case CS_METRIC_MIN_S2: metric = c > 0.f ? st.mn[i] : INFINITY; break;
                    default:
                        metric = c > 0.f ? st.sm_m[i] - k.tau * 0.6931471805599453f * lg2_approx(st.sm_acc[i])
                                         : INFINITY;
                }
            }
            if (a.out_metric) a.out_metric[row] = metric;
            if (a.out_collide) a.out_collide[row] = col;
            if (a.out_count) a.out_count[row] = cntv;
        } else {
            float gxo = 0.f, gyo = 0.f, gzo = 0.f;
            if (!valid[i] || !ok) {
                gxo = gyo = gzo = __int_as_float(0x7fc00000);
            } else {
                const float c = st.cnt[i];
                nb_total += c;
                float up = 1.f;
                if (a.grad_out) up = a.grad_out[k.group_size > 0 ? row / (uint32_t)k.group_size : row];
                float f = 0.f;
                switch (k.mode) {
                    case CS_METRIC_MEAN_COST: f = c > 0.f ? -k.gamma * k.d_max / c : 0.f; break;
                    case CS_METRIC_SUM_COST: f = -k.gamma * k.d_max; break;
                    case CS_METRIC_MIN_S2: f = c > 0.f ? 1.f : 0.f; break;
                    default: f = c > 0.f ? 1.f / st.sm_acc[i] : 0.f;
                }
                f *= up;
                gxo = st.gx[i] * f; gyo = st.gy[i] * f; gzo = st.gz[i] * f;
            }
            a.grad_centres[3 * (size_t)row + 0] = gxo;
            a.grad_centres[3 * (size_t)row + 1] = gyo;
            a.grad_centres[3 * (size_t)row + 2] = gzo;
        }
    }
    if (a.stats) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nb_total += __shfl_xor_sync(0xffffffffu, nb_total, o);
        if (lane == 0) {
            atomicAdd(a.stats + 0, (unsigned long long)evaluated * (unsigned long long)nvalid);
            atomicAdd(a.stats + 1, (unsigned long long)nb_total);
        }
    }
}

template <int PRIM, int QB, int NCW, bool SOFTMIN, bool GRAD>
__global__ void __launch_bounds__((NCW + 1) * 32) k_eval(const EvalArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EvalSmem *sm = reinterpret_cast<EvalSmem *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], NCW);
        }
        fence_mbar_init();
        sm->abort = (*(volatile unsigned *)a.err & kErrTimeout) ? 1 : 0;
    }
    __syncthreads();
    const int tile = blockIdx.x;
    const bool abort = sm->abort != 0;
    if (warp == NCW) {
        if (!abort) producer_warp<PRIM, QB, NCW>(a, sm, tile);
    } else {
        consumer_warp<PRIM, QB, NCW, SOFTMIN, GRAD>(a, sm, tile, warp, abort);
    }
}

// ------------------------------------------------------ preparation kernels
__device__ __forceinline__ uint32_t spread8(uint32_t v) {
    v &= 0xFFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Morton key of each primitive centre over the scene box (8 bits per axis).
__global__ void k_prep_keys(const float *__restrict__ prims, int stride, int Q, SceneDev sc,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Q) return;
    const float *p = prims + (size_t)j * stride;
    uint32_t code = 0;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (p[a] - sc.bb_lo[a]) / (sc.bb_hi[a] - sc.bb_lo[a]) * 256.f;
        u = isfinite(u) ? fminf(fmaxf(u, 0.f), 255.f) : 255.f;
        c[a] = (uint32_t)u;
    }
    code = spread8(c[0]) | (spread8(c[1]) << 1) | (spread8(c[2]) << 2);
    keys[j] = code;
    vals[j] = (uint32_t)j;
}

// Prepared records in sorted order.  Sphere: (c, r).  Ellipsoid:
// (c, a_max), (Axx, Ayy, Azz, Axy), (Axz, Ayz, a_min, 0) with
// A = R diag(1/a^2, 1/b^2, 1/c^2) R^T (Eq. 6).  Invalid rows get w = NaN.
__global__ void k_prep_recs(const float *__restrict__ prims, int prim_type, int Q,
                            const uint32_t *__restrict__ perm, float ns_scalar,
                            const float *__restrict__ ns_rows, float4 *__restrict__ qrec,
                            float *__restrict__ qns, unsigned *__restrict__ err) {
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= Q) return;
    const uint32_t j = perm[q];
    float ns = ns_rows ? ns_rows[j] : ns_scalar;
    bool ok = isfinite(ns) && ns >= 0.f;
    const float nanf_ = __int_as_float(0x7fc00000);
    if (prim_type == CS_PRIM_SPHERE) {
        const float *pp = prims + (size_t)j * 4;
        float4 p = make_float4(pp[0], pp[1], pp[2], pp[3]);
        ok = ok && isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(p.w) && p.w > 0.f;
        qrec[q] = make_float4(p.x, p.y, p.z, ok ? p.w : nanf_);
    } else {
        const float *p = prims + (size_t)j * 10;
        float cx = p[0], cy = p[1], cz = p[2], qw = p[3], qx = p[4], qy = p[5], qz = p[6];
        float ea = p[7], eb = p[8], ec = p[9];
        ok = ok && isfinite(cx) && isfinite(cy) && isfinite(cz) && isfinite(qw) && isfinite(qx) &&
             isfinite(qy) && isfinite(qz) && isfinite(ea) && isfinite(eb) && isfinite(ec) &&
             ea > 0.f && eb > 0.f && ec > 0.f;
        float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
        if (!(n2 > 0.f)) { qw = 1.f; qx = qy = qz = 0.f; n2 = 1.f; }
        float s = 2.f / n2;
        float R00 = 1.f - s * (qy * qy + qz * qz), R01 = s * (qx * qy - qw * qz), R02 = s * (qx * qz + qw * qy);
        float R10 = s * (qx * qy + qw * qz), R11 = 1.f - s * (qx * qx + qz * qz), R12 = s * (qy * qz - qw * qx);
        float R20 = s * (qx * qz - qw * qy), R21 = s * (qy * qz + qw * qx), R22 = 1.f - s * (qx * qx + qy * qy);
        float p0 = 1.f / (ea * ea), p1 = 1.f / (eb * eb), p2 = 1.f / (ec * ec);
        float Axx = R00 * R00 * p0 + R01 * R01 * p1 + R02 * R02 * p2;
        float Ayy = R10 * R10 * p0 + R11 * R11 * p1 + R12 * R12 * p2;
        float Azz = R20 * R20 * p0 + R21 * R21 * p1 + R22 * R22 * p2;
        float Axy = R00 * R10 * p0 + R01 * R11 * p1 + R02 * R12 * p2;
        float Axz = R00 * R20 * p0 + R01 * R21 * p1 + R02 * R22 * p2;
        float Ayz = R10 * R20 * p0 + R11 * R21 * p1 + R12 * R22 * p2;
        float amax = fmaxf(fmaxf(ea, eb), ec), amin = fminf(fminf(ea, eb), ec);
        qrec[3 * (size_t)q + 0] = make_float4(cx, cy, cz, ok ? amax : nanf_);
        qrec[3 * (size_t)q + 1] = make_float4(Axx, Ayy, Azz, Axy);
        qrec[3 * (size_t)q + 2] = make_float4(Axz, Ayz, amin, 0.f);
    }
    qns[q] = ok ? ns : 0.f;
    if (!ok) atomicOr(err, kErrInvalidQuery);
}

// Section II-D/E group outputs: metric summed, flag OR-ed over runs of G rows.
__global__ void k_group(const float *__restrict__ metric, const uint8_t *__restrict__ collide,
                        int Q, int G, float *__restrict__ gm, uint8_t *__restrict__ gc) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    int ng = (Q + G - 1) / G;
    if (g >= ng) return;
    int b = g * G, e = min(Q, b + G);
    float s = 0.f;
    uint8_t c = 0;
    for (int j = b; j < e; ++j) {
        if (metric) s += metric[j];
        if (collide) c |= collide[j];
    }
    if (gm) gm[g] = s;
    if (gc) gc[g] = c;
}

// ---------------------------------------------------------- host launchers
QueryConsts make_consts(const cs_params &p) {
    QueryConsts k;
    const double S_cut = (double)p.s_min + log(1.0 / (double)p.eps) / (double)p.gamma;
    k.S_cut = (float)S_cut;
    k.S_reach = (float)std::max(S_cut, 1.0);
    k.T_in = S_cut >= 1.0 ? 1.f : nextafterf(k.S_cut, INFINITY);
    k.G = (float)((double)p.gamma * 1.4426950408889634);
    k.Gsmin = (float)((double)p.gamma * 1.4426950408889634 * (double)p.s_min);
    k.s_min = p.s_min;
    k.d_max = p.d_max;
    k.gamma = p.gamma;
    k.tau = p.tau;
    k.K = (float)(1.0 / ((double)p.tau * 0.6931471805599453));
    k.k_thr = p.k_thr;
    k.mode = p.mode;
    k.group_size = p.group_size;
    return k;
}


struct TileCfg {
    int id;
    int qb;
};
// ids: 1 = 1 primitive per lane (128 per tile), 2 = 2 (256), 3 = 4 (512)
static const TileCfg kTileCfgs[] = {{1, 1}, {2, 2}, {3, 4}};

int tile_configs(int32_t *ids, int32_t cap) {
    int n = (int)(sizeof(kTileCfgs) / sizeof(kTileCfgs[0]));
    for (int i = 0; i < n && i < cap; ++i) ids[i] = kTileCfgs[i].id;
    return n;
}

constexpr int kNCW = 4;

template <int PRIM, int QB, bool SOFTMIN, bool GRAD>
static cudaError_t launch_eval_t(const EvalArgs &a, cudaStream_t s) {
    constexpr int TQ = kNCW * 32 * QB;
    const int ntiles = (a.Q + TQ - 1) / TQ;
    static_assert(sizeof(EvalSmem) <= 48 * 1024, "stage ring must fit the default smem limit");
    k_eval<PRIM, QB, kNCW, SOFTMIN, GRAD><<<ntiles, (kNCW + 1) * 32, sizeof(EvalSmem), s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

template <int PRIM, int QB>
static cudaError_t launch_eval_qb(const EvalArgs &a, bool grad, cudaStream_t s) {
    const bool soft = a.k.mode == CS_METRIC_SOFTMIN_S2;
    if (grad) return launch_eval_t<PRIM, QB, false, true>(a, s);
    if (soft) return launch_eval_t<PRIM, QB, true, false>(a, s);
    return launch_eval_t<PRIM, QB, false, false>(a, s);
}

static int choose_qb(int prim_type, int Q, int tile_cfg, int num_sms) {
    for (const TileCfg &t : kTileCfgs)
        if (t.id == tile_cfg) return (prim_type == CS_PRIM_ELLIPSOID && t.qb > 2) ? 2 : t.qb;
    // automatic: the largest tile that still gives every SM four tiles
    const int cand[3] = {4, 2, 1};
    for (int qb : cand) {
        if (prim_type == CS_PRIM_ELLIPSOID && qb > 2) continue;
        int ntiles = (Q + kNCW * 32 * qb - 1) / (kNCW * 32 * qb);
        if (ntiles >= 4 * num_sms) return qb;
    }
    return 1;
}

cudaError_t launch_eval(int prim_type, const EvalArgs &a, bool grad, int tile_cfg, int num_sms,
                        cudaStream_t s) {
    int qb = choose_qb(prim_type, a.Q, tile_cfg, num_sms);
    if (prim_type == CS_PRIM_SPHERE) {
        if (qb == 4) return launch_eval_qb<0, 4>(a, grad, s);
        if (qb == 2) return launch_eval_qb<0, 2>(a, grad, s);
        return launch_eval_qb<0, 1>(a, grad, s);
    }
    if (qb == 2) return launch_eval_qb<1, 2>(a, grad, s);
    return launch_eval_qb<1, 1>(a, grad, s);
}

cudaError_t run_eval(int prim_type, const SceneDev &sc, const float4 *qrec, const float *qns,
                     const uint32_t *perm, int Q, const cs_params &p, float *out_metric,
                     uint8_t *out_collide, int32_t *out_count, const float *grad_out,
                     float *grad_centres, unsigned *err, int num_sms, long long polls,
                     cudaStream_t s) {
    EvalArgs a;
    a.sc = sc;
    a.qrec = qrec;
    a.qns = qns;
    a.perm = perm;
    a.Q = Q;
    a.k = make_consts(p);
    a.out_metric = out_metric;
    a.out_collide = out_collide;
    a.out_count = out_count;
    a.grad_out = grad_out;
    a.grad_centres = grad_centres;
    a.err = err;
    a.stats = p.out_pair_stats;
    a.wait_polls = polls;
    cudaError_t e;
    if (p.eval_events[0] && (e = cudaEventRecord((cudaEvent_t)p.eval_events[0], s)) != cudaSuccess) return e;
    e = launch_eval(prim_type, a, grad_centres != nullptr, p.tile_config, num_sms, s);
    if (e == cudaSuccess && p.eval_events[1]) e = cudaEventRecord((cudaEvent_t)p.eval_events[1], s);
    return e;
}

// One block waits on a barrier that nothing completes; the bounded wait must
// give up and record the timeout.
__global__ void k_wait_selftest(long long polls, unsigned *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!wait_phase(&bar, 0u, polls)) atomicOr(err, kErrTimeout);
    }
}

cudaError_t run_wait_selftest(long long polls, unsigned *err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(polls, err);
    count_launches(1);
    return cudaGetLastError();
}

void launch_prep(const float *prims, int prim_type, int Q, const SceneDev &sc, float ns_scalar,
                 const float *ns_rows, Workspace &ws, uint32_t **perm_out, cudaStream_t s) {
    const int stride = prim_type == CS_PRIM_SPHERE ? 4 : 10;
    const int thr = 256, blk = (Q + thr - 1) / thr;
    k_prep_keys<<<blk, thr, 0, s>>>(prims, stride, Q, sc, ws.keys[0], ws.vals[0]);
    count_launches(1);
    int res = radix_sort(ws.keys, ws.vals, (size_t)Q, 3 * kMortonBits, ws.sort_hist, ws.scan_tmp, s);
    uint32_t *perm = ws.vals[res];
    k_prep_recs<<<blk, thr, 0, s>>>(prims, prim_type, Q, perm, ns_scalar, ns_rows, ws.qrec,
                                    ws.qns, ws.err);
    count_launches(1);
    *perm_out = perm;
}

void launch_group(const float *metric, const uint8_t *collide, int Q, int G, float *gm, uint8_t *gc,
                  cudaStream_t s) {
    int ng = (Q + G - 1) / G;
    k_group<<<(ng + 255) / 256, 256, 0, s>>>(metric, collide, Q, G, gm, gc);
    count_launches(1);
}

}  // namespace cs
