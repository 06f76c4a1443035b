// cs_render.cu -- image synthesis of Section II-A (Eq. 3-4) over the resident
// scene: the terminal-state images of Section II-D, rendered in batches of
// views into device buffers.
//
// Pipeline for V views of a scene with S slots (32 per chunk):
//   k_rs_project   one warp per (view, chunk), lane = slot: the mean's
//                  projection, Sigma' (Eq. 3) and its inverse, the float32
//                  depth key, and the range of 16x16 tiles the footprint
//                  alpha G >= 1/255 can touch (a chunk whose means all lie
//                  behind the near plane is skipped whole);
//   scan           exclusive scan of the per-(view, slot) tile counts;
//   k_rs_emit      one instance per (view, Gaussian, tile);
//   radix sorts    stable: by depth bits, then by view * tiles + tile, giving
//                  each tile's list front to back (equal depths in slot order);
//   k_rs_ranges    each tile's run in the sorted list;
//   k_rs_render    one CTA per (view, tile), one thread per pixel: batches of
//                  256 projected Gaussians staged in shared memory, blended
//                  front to back (Eq. 4) until every pixel of the tile stops.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <algorithm>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kTile = 16;                              // tile edge in pixels
constexpr float kAlphaMin = 1.f / 255.f;               // smallest alpha G that counts
constexpr float kAlphaMax = 0.99f;                     // clamp of alpha G
constexpr float kTransMin = 1e-4f;                     // a pixel stops below this transmittance
constexpr float kHalfLog2e = 0.72134752044448170368f;  // exp(-q/2) = 2^(-q * kHalfLog2e)

struct RenderConsts {
    int W, H, tiles_x, tiles_y, T, V;
    int nchunks;
    uint32_t S;  // slots per view
    float near_plane, dilation;
    float bg[3];
};

// Projected Gaussian, three float4 per (view, slot):
//   (u, v, pa, pb) (pc, opacity, distance, x range) (r, g, b, y range)
// with 2^-(pa dx^2 + pb dx dy + pc dy^2) = G2D at offset (dx, dy), and the
// pixel columns / rows its footprint can touch packed as lo | hi << 16; the
// float32 depth (the sort key) goes to its own array.
__global__ void __launch_bounds__(256) k_rs_project(SceneDev sc, const float4 *__restrict__ app,
                                                    const cs_camera *__restrict__ cams, RenderConsts rc,
                                                    float4 *__restrict__ proj, float *__restrict__ zkey,
                                                    uint32_t *__restrict__ ntile,
                                                    unsigned long long *__restrict__ total) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int v = blockIdx.y;
    if (c >= rc.nchunks) return;  // whole warps
    const float *cf = reinterpret_cast<const float *>(cams + v);
    const float r0 = __ldg(cf + 0), r1 = __ldg(cf + 1), r2 = __ldg(cf + 2), r3 = __ldg(cf + 3), r4 = __ldg(cf + 4),
                r5 = __ldg(cf + 5), r6 = __ldg(cf + 6), r7 = __ldg(cf + 7), r8 = __ldg(cf + 8);
    const float t0 = __ldg(cf + 9), t1 = __ldg(cf + 10), t2 = __ldg(cf + 11);
    const float fx = __ldg(cf + 12), fy = __ldg(cf + 13), cx = __ldg(cf + 14), cy = __ldg(cf + 15);
    const ChunkBlock &B = sc.blocks[c];
    const size_t g = (size_t)v * rc.S + (size_t)c * kChunk + lane;
    const float4 lo = B.lo, hi = B.hi;
    // largest camera depth of the chunk's box, padded for rounding
    const float mx = 0.5f * (lo.x + hi.x), my = 0.5f * (lo.y + hi.y), mz = 0.5f * (lo.z + hi.z);
    const float ex = 0.5f * (hi.x - lo.x), ey = 0.5f * (hi.y - lo.y), ez = 0.5f * (hi.z - lo.z);
    const float zc = fmaf(r8, mz, fmaf(r7, my, r6 * mx)) + t2;
    const float ze = fmaf(fabsf(r8), ez, fmaf(fabsf(r7), ey, fabsf(r6) * ex));
    uint32_t n = 0;
    const bool chunk_live = zc + ze + 1e-4f * (fabsf(zc) + ze) + 1e-6f >= rc.near_plane;
    if (chunk_live && lane < (int)hi.w) {
        const float4 ap = app[(size_t)c * kChunk + lane];
        const float x = B.x[lane], y = B.y[lane], z = B.z[lane];
        // the sort key: rounded after every operation, in this order
        const float zz = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r6, x), __fmul_rn(r7, y)), __fmul_rn(r8, z)), t2);
        if (ap.x >= kAlphaMin && zz >= rc.near_plane) {
            const float xc = fmaf(r2, z, fmaf(r1, y, r0 * x)) + t0;
            const float yc = fmaf(r5, z, fmaf(r4, y, r3 * x)) + t1;
            const float iz = 1.f / zz;
            const float u = fmaf(fx * xc, iz, cx), vv = fmaf(fy * yc, iz, cy);
            // J = d(u, v)/d(x_c) at the mean, M = J R (Eq. 3)
            const float j00 = fx * iz, j11 = fy * iz;
            const float j02 = -j00 * xc * iz, j12 = -j11 * yc * iz;
            const float m00 = fmaf(j02, r6, j00 * r0), m01 = fmaf(j02, r7, j00 * r1), m02 = fmaf(j02, r8, j00 * r2);
            const float m10 = fmaf(j12, r6, j11 * r3), m11 = fmaf(j12, r7, j11 * r4), m12 = fmaf(j12, r8, j11 * r5);
            const float sxx = B.sxx[lane], syy = B.syy[lane], szz = B.szz[lane];
            const float sxy = 0.5f * B.sxy2[lane], sxz = 0.5f * B.sxz2[lane], syz = 0.5f * B.syz2[lane];
            const float a0 = fmaf(sxz, m02, fmaf(sxy, m01, sxx * m00));
            const float a1 = fmaf(syz, m02, fmaf(syy, m01, sxy * m00));
            const float a2 = fmaf(szz, m02, fmaf(syz, m01, sxz * m00));
            const float b0 = fmaf(sxz, m12, fmaf(sxy, m11, sxx * m10));
            const float b1 = fmaf(syz, m12, fmaf(syy, m11, sxy * m10));
            const float b2 = fmaf(szz, m12, fmaf(syz, m11, sxz * m10));
            const float A = fmaf(m02, a2, fmaf(m01, a1, m00 * a0)) + rc.dilation;  // Sigma'_xx
            const float Bc = fmaf(m12, a2, fmaf(m11, a1, m10 * a0));                // Sigma'_xy
            const float C = fmaf(m12, b2, fmaf(m11, b1, m10 * b0)) + rc.dilation;   // Sigma'_yy
            const float det = fmaf(A, C, -(Bc * Bc));
            if (det > 0.f) {
                // footprint: alpha G >= 1/255 <=> q <= 2 ln(255 alpha); its box has
                // half-extents sqrt(q Sigma'_xx), sqrt(q Sigma'_yy).  The box is
                // widened by the FP32 error of q and of Sigma' (relative, at most
                // ~40 u kappa with kappa the condition number of Sigma'), so every
                // pixel the blending can draw lies inside it.
                const float tr = 0.5f * (A + C), disc = sqrtf(fmaf(0.25f * (A - C), A - C, Bc * Bc));
                const float lmax = tr + disc, kap = lmax * lmax / det;  // lmax / lmin, lmin = det / lmax
                const float grow = fmaf(40.f * 5.9604645e-8f, kap, 1.0001f);
                const float qmax = fmaxf(2.f * logf(255.f * ap.x), 0.f);
                const float rx = fmaf(sqrtf(qmax * A), grow, 1e-3f), ry = fmaf(sqrtf(qmax * C), grow, 1e-3f);
                // pixel i is touched when |i + 0.5 - u| <= rx
                const float fx0 = fmaxf(ceilf(u - rx - 0.5f), 0.f), fx1 = fminf(floorf(u + rx - 0.5f), (float)(rc.W - 1));
                const float fy0 = fmaxf(ceilf(vv - ry - 0.5f), 0.f), fy1 = fminf(floorf(vv + ry - 0.5f), (float)(rc.H - 1));
                if (fx0 <= fx1 && fy0 <= fy1) {
                    const uint32_t x0 = (uint32_t)fx0, x1 = (uint32_t)fx1, y0 = (uint32_t)fy0, y1 = (uint32_t)fy1;
                    n = ((x1 >> 4) - (x0 >> 4) + 1) * ((y1 >> 4) - (y0 >> 4) + 1);
                    const float id = 1.f / det;
                    const float dist = sqrtf(fmaf(zz, zz, fmaf(yc, yc, xc * xc)));
                    proj[3 * g + 0] = make_float4(u, vv, C * id * kHalfLog2e, -2.f * Bc * id * kHalfLog2e);
                    proj[3 * g + 1] = make_float4(A * id * kHalfLog2e, ap.x, dist, __uint_as_float(x0 | (x1 << 16)));
                    proj[3 * g + 2] = make_float4(ap.y, ap.z, ap.w, __uint_as_float(y0 | (y1 << 16)));
                    zkey[g] = zz;
                }
            }
        }
    }
    ntile[g] = n;
    unsigned long long tot = n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) atomicAdd(total, tot);
}

// One instance per (view, Gaussian, tile), in (view, slot, tile) order.
__global__ void k_rs_emit(const float4 *__restrict__ proj, const float *__restrict__ zkey,
                          const uint32_t *__restrict__ ntile, const uint32_t *__restrict__ offs, RenderConsts rc,
                          size_t VS,
                          uint32_t *__restrict__ dkey, uint32_t *__restrict__ ival, uint32_t *__restrict__ tkey,
                          uint32_t *__restrict__ iproj) {
    const size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= VS) return;
    const uint32_t n = ntile[g];
    if (n == 0) return;
    const uint32_t base = offs[g];
    const uint32_t zbits = __float_as_uint(zkey[g]);
    const uint32_t xr = __float_as_uint(proj[3 * g + 1].w), yr = __float_as_uint(proj[3 * g + 2].w);
    const uint32_t tx0 = (xr & 0xFFFFu) >> 4, tx1 = (xr >> 16) >> 4, ty0 = (yr & 0xFFFFu) >> 4, ty1 = (yr >> 16) >> 4;
    const uint32_t tbase = (uint32_t)(g / rc.S) * (uint32_t)rc.T;
    uint32_t i = base;
    for (uint32_t ty = ty0; ty <= ty1; ++ty)
        for (uint32_t tx = tx0; tx <= tx1; ++tx, ++i) {
            dkey[i] = zbits;
            ival[i] = i;
            tkey[i] = tbase + ty * (uint32_t)rc.tiles_x + tx;
            iproj[i] = (uint32_t)g;
        }
}

__global__ void k_rs_gather(const uint32_t *__restrict__ idx, const uint32_t *__restrict__ src, uint32_t n,
                            uint32_t *__restrict__ dst) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// Each tile's run [x, y) in the sorted instances, and the projection index of
// every sorted instance.
__global__ void k_rs_ranges(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ inst,
                            const uint32_t *__restrict__ iproj, uint32_t n, uint2 *__restrict__ ranges,
                            uint32_t *__restrict__ spidx) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t t = tkeys[i];
    if (i == 0 || tkeys[i - 1] != t) ranges[t].x = i;
    if (i == n - 1 || tkeys[i + 1] != t) ranges[t].y = i + 1;
    spidx[i] = iproj[inst[i]];
}

// One CTA per (tile, view), one thread per pixel: Eq. 4 front to back.
__global__ void __launch_bounds__(256) k_rs_render(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ spidx,
                                                   const float4 *__restrict__ proj, RenderConsts rc,
                                                   float *__restrict__ rgb, float *__restrict__ depth,
                                                   float *__restrict__ alpha) {
    __shared__ float4 s0[256], s1[256], s2[256];
    const int tile = blockIdx.x, v = blockIdx.y;
    const int tx = tile % rc.tiles_x, ty = tile / rc.tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1)), py = ty * kTile + (threadIdx.x >> 4);
    const bool inside = px < rc.W && py < rc.H;
    const uint2 r = ranges[(size_t)v * rc.T + tile];
    const float fx = (float)px + 0.5f, fy = (float)py + 0.5f;
    const uint32_t row0 = (uint32_t)(ty * kTile + 2 * (threadIdx.x >> 5));  // this warp's two rows
    float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, dd = 0.f;
    bool done = !inside;
    for (uint32_t start = r.x; start < r.y; start += 256) {
        if (__syncthreads_count(done) == 256) break;
        const uint32_t i = start + threadIdx.x;
        if (i < r.y) {
            const size_t id = spidx[i];
            s0[threadIdx.x] = proj[3 * id];
            s1[threadIdx.x] = proj[3 * id + 1];
            s2[threadIdx.x] = proj[3 * id + 2];
        }
        __syncthreads();
        const int n = (int)min(256u, r.y - start);
        if (!done) {
            for (int k = 0; k < n; ++k) {
                const float4 c2 = s2[k];
                // the whole warp skips a Gaussian whose footprint misses its two rows
                const uint32_t yr = __float_as_uint(c2.w);
                if ((yr & 0xFFFFu) > row0 + 1 || (yr >> 16) < row0) continue;
                const float4 a = s0[k], b = s1[k];
                const float dx = fx - a.x, dy = fy - a.y;
                const float power = fmaf(a.z, dx * dx, fmaf(a.w, dx * dy, b.x * (dy * dy)));
                const float A = b.y * ex2_approx(-power);
                if (A < kAlphaMin) continue;
                const float al = fminf(A, kAlphaMax);
                const float Tn = T * (1.f - al);
                if (Tn < kTransMin) {
                    done = true;
                    break;
                }
                const float w = al * T;
                cr = fmaf(w, c2.x, cr);
                cg = fmaf(w, c2.y, cg);
                cb = fmaf(w, c2.z, cb);
                dd = fmaf(w, b.z, dd);
                T = Tn;
            }
        }
        __syncthreads();
    }
    if (!inside) return;
    const size_t p = ((size_t)v * rc.H + py) * rc.W + px;
    rgb[3 * p + 0] = fmaf(T, rc.bg[0], cr);
    rgb[3 * p + 1] = fmaf(T, rc.bg[1], cg);
    rgb[3 * p + 2] = fmaf(T, rc.bg[2], cb);
    if (depth) depth[p] = dd;
    if (alpha) alpha[p] = 1.f - T;
}

// Appearance into slot order; padding slots keep opacity 0.
__global__ void k_rs_appearance(const int32_t *__restrict__ index, const int32_t *__restrict__ slot_of, int n,
                                const float *__restrict__ op, const float *__restrict__ col,
                                float4 *__restrict__ app) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = index[p];
    const float o = op ? op[i] : 1.f;
    const float r = col ? col[3 * (size_t)i] : 1.f, g = col ? col[3 * (size_t)i + 1] : 1.f,
                b = col ? col[3 * (size_t)i + 2] : 1.f;
    app[slot_of[p]] = make_float4(o, r, g, b);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Grow a scratch buffer to at least `need` bytes (by half again its old size
// at least, so a slowly growing workload reallocates rarely).
cs_status ensure(void **buf, size_t *cap, size_t need) {
    if (*cap >= need) return CS_OK;
    const size_t grow = std::max(need, *cap + *cap / 2);
    if (*buf) CS_CUDA(cudaFree(*buf));
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, grow);
    if (e != cudaSuccess) {
        *buf = nullptr;
        if (e == cudaErrorMemoryAllocation) {
            (void)cudaGetLastError();
            set_error("render scratch allocation failed");
            return CS_ERR_NO_MEMORY;
        }
        return cuda_fail(e, "cudaMalloc(render scratch)");
    }
    *cap = grow;
    return CS_OK;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" {

cs_status cs_render_desc_init(cs_render_desc *d) {
    if (!d) return invalid("desc is NULL");
    memset(d, 0, sizeof(*d));
    d->near_plane = 0.01f;
    d->dilation = 0.3f;
    return CS_OK;
}

cs_status cs_scene_set_appearance(cs_scene *scene, const float *opacity, const float *colors, int32_t on_device,
                                  void *stream) {
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (on_device != 0 && on_device != 1) return invalid("on_device must be 0 or 1");
    Scene *sc = reinterpret_cast<Scene *>(scene);
    cudaStream_t s = (cudaStream_t)stream;
    const SceneDev &dv = sc->dev;
    const size_t slots = (size_t)std::max(dv.nchunks, 1) * kChunk;
    if (!sc->app) {
        cudaError_t e = cudaMalloc(&sc->app, sizeof(float4) * slots);
        if (e != cudaSuccess) {
            sc->app = nullptr;
            return cuda_fail(e, "cudaMalloc(appearance)");
        }
    }
    CS_CUDA(cudaMemsetAsync(sc->app, 0, sizeof(float4) * slots, s));
    const float *op = opacity, *col = colors;
    void *tmp = nullptr;
    const int64_t n = sc->n_input;
    if (!on_device && n > 0 && (opacity || colors)) {
        CS_CUDA(cudaMalloc(&tmp, 16 * (size_t)n));
        float *t = (float *)tmp;
        if (opacity) {
            CS_CUDA(cudaMemcpyAsync(t, opacity, 4 * (size_t)n, cudaMemcpyHostToDevice, s));
            op = t;
        }
        if (colors) {
            CS_CUDA(cudaMemcpyAsync(t + n, colors, 12 * (size_t)n, cudaMemcpyHostToDevice, s));
            col = t + n;
        }
    }
    if (dv.n_gauss > 0) {
        k_rs_appearance<<<(dv.n_gauss + 255) / 256, 256, 0, s>>>(dv.index, dv.slot_of, dv.n_gauss, op, col, sc->app);
        count_launches(1);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "cs_scene_set_appearance");
    return CS_OK;
}

cs_status cs_render(const cs_scene *scene, const cs_render_desc *d, const cs_camera *cams, float *out_rgb,
                    float *out_depth, float *out_alpha) {
    NvtxRange range("cs.render");
    cs_status st = check_scene(scene);
    if (st != CS_OK) return st;
    if (!d) return invalid("desc is NULL");
    if (d->n_views < 0 || d->n_views > 65535) return invalid("n_views must lie in [0, 65535]");
    if (d->width < 1 || d->width > 4096 || d->height < 1 || d->height > 4096)
        return invalid("width and height must lie in [1, 4096]");
    if (!(d->near_plane >= 0.f) || !isfinite(d->near_plane)) return invalid("near_plane must be finite and >= 0");
    if (!(d->dilation >= 0.f) || !isfinite(d->dilation)) return invalid("dilation must be finite and >= 0");
    for (int k = 0; k < 3; ++k)
        if (!isfinite(d->background[k])) return invalid("background must be finite");
    const Scene *sc = reinterpret_cast<const Scene *>(scene);
    if (!sc->app) return invalid("the scene has no appearance: call cs_scene_set_appearance first");
    if (d->n_views == 0) return CS_OK;
    if (!cams || !out_rgb) return invalid("cams and out_rgb are required");
    cudaStream_t s = (cudaStream_t)d->stream;
    const SceneDev &dv = sc->dev;

    RenderConsts rc;
    rc.W = d->width;
    rc.H = d->height;
    rc.tiles_x = (d->width + kTile - 1) / kTile;
    rc.tiles_y = (d->height + kTile - 1) / kTile;
    rc.T = rc.tiles_x * rc.tiles_y;
    rc.V = d->n_views;
    rc.nchunks = dv.nchunks;
    rc.S = (uint32_t)dv.nchunks * kChunk;
    rc.near_plane = d->near_plane;
    rc.dilation = d->dilation;
    for (int k = 0; k < 3; ++k) rc.bg[k] = d->background[k];
    const size_t VT = (size_t)rc.V * rc.T;
    int tbits = 8;
    while (tbits < 32 && ((size_t)1 << tbits) < VT) tbits += 8;
    const size_t VS = (size_t)rc.V * rc.S;
    if (VS >= ((size_t)1 << 32)) {
        set_error("more than 2^32 (view, Gaussian slot) pairs: render fewer views per call");
        return CS_ERR_UNSUPPORTED;
    }

    Workspace *w = nullptr;
    if ((st = get_workspace(sc->device, s, 1, false, &w)) != CS_OK) return st;
    // per (view, slot): projections, tile counts, their scan, the instance total
    const size_t o_zkey = align256(48 * VS), o_ntile = align256(o_zkey + 4 * VS), o_offs = align256(o_ntile + 4 * VS);
    const size_t o_total = align256(o_offs + 4 * VS);
    const size_t o_scan = align256(o_total + 8);
    const size_t need1 = o_scan + 4 * scan_tmp_elems(std::max<size_t>(VS, 1));
    if ((st = ensure(&w->rnd, &w->cap_rnd, need1)) != CS_OK) return st;
    char *b1 = (char *)w->rnd;
    float4 *proj = (float4 *)b1;
    float *zkey = (float *)(b1 + o_zkey);
    uint32_t *ntile = (uint32_t *)(b1 + o_ntile), *offs = (uint32_t *)(b1 + o_offs);
    unsigned long long *total = (unsigned long long *)(b1 + o_total);
    uint32_t *scan1 = (uint32_t *)(b1 + o_scan);
    CS_CUDA(cudaMemsetAsync(total, 0, 8, s));
    if (VS > 0) {
        k_rs_project<<<dim3((unsigned)((rc.nchunks + 7) / 8), (unsigned)rc.V), 256, 0, s>>>(dv, sc->app, cams, rc, proj,
                                                                                          zkey, ntile, total);
        count_launches(1);
        CS_CUDA(cudaGetLastError());
        scan_exclusive(ntile, offs, VS, scan1, s);
    }
    unsigned long long I64 = 0;
    CS_CUDA(cudaMemcpyAsync(&I64, total, 8, cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    if (I64 > ((unsigned long long)1 << 31)) {
        set_error("more than 2^31 (view, Gaussian, tile) instances: render fewer views per call");
        return CS_ERR_UNSUPPORTED;
    }
    const size_t I = (size_t)I64;
    if (d->out_instances) *d->out_instances = (int64_t)I64;

    // per instance: two key and two value buffers, tile keys, projection
    // indices (unsorted and sorted), tile ranges, sort scratch
    const size_t n4 = align256(4 * std::max<size_t>(I, 1));
    const size_t hist_n = sort_hist_elems(std::max<size_t>(I, 1));
    const size_t o_ranges = 7 * n4, o_hist = align256(o_ranges + 8 * VT), o_scan2 = align256(o_hist + 4 * hist_n);
    const size_t need2 = o_scan2 + 4 * scan_tmp_elems(hist_n);
    if ((st = ensure(&w->rnd2, &w->cap_rnd2, need2)) != CS_OK) return st;
    char *b2 = (char *)w->rnd2;
    uint32_t *dkey[2] = {(uint32_t *)b2, (uint32_t *)(b2 + n4)};
    uint32_t *ival[2] = {(uint32_t *)(b2 + 2 * n4), (uint32_t *)(b2 + 3 * n4)};
    uint32_t *tkey = (uint32_t *)(b2 + 4 * n4), *iproj = (uint32_t *)(b2 + 5 * n4), *spidx = (uint32_t *)(b2 + 6 * n4);
    uint2 *ranges = (uint2 *)(b2 + o_ranges);
    uint32_t *hist = (uint32_t *)(b2 + o_hist), *scan2 = (uint32_t *)(b2 + o_scan2);
    CS_CUDA(cudaMemsetAsync(ranges, 0, 8 * VT, s));
    if (I > 0) {
        k_rs_emit<<<(unsigned)((VS + 255) / 256), 256, 0, s>>>(proj, zkey, ntile, offs, rc, VS, dkey[0], ival[0],
                                                               tkey, iproj);
        count_launches(1);
        const int r1 = radix_sort(dkey, ival, I, 32, hist, scan2, s);
        k_rs_gather<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(ival[r1], tkey, (uint32_t)I, dkey[r1 ^ 1]);
        count_launches(1);
        uint32_t *k2[2] = {dkey[r1 ^ 1], dkey[r1]};
        uint32_t *v2[2] = {ival[r1], ival[r1 ^ 1]};
        const int r2 = radix_sort(k2, v2, I, tbits, hist, scan2, s);
        k_rs_ranges<<<(unsigned)((I + 255) / 256), 256, 0, s>>>(k2[r2], v2[r2], iproj, (uint32_t)I, ranges, spidx);
        count_launches(1);
    }
    k_rs_render<<<dim3((unsigned)rc.T, (unsigned)rc.V), 256, 0, s>>>(ranges, spidx, proj, rc, out_rgb, out_depth,
                                                                    out_alpha);
    count_launches(1);
    CS_CUDA(cudaGetLastError());
    return CS_OK;
}

}  // extern "C"
