// cs_build.cu -- scene construction: Eq. 2 repack of every Gaussian, the
// floater filter of Section II-C, and the spatial index the cull descends (the
// paper uses a spatial hash, Section II-B): Gaussians in global Hilbert-curve
// order of their means, a separate tier for the very large ones, chunks of up to 32
// consecutive Gaussians within an extent limit, and a fan-out-32 tree of
// bounding records over the chunks.
#include <math.h>

#include <algorithm>
#include <vector>

#include "cs_internal.cuh"

namespace cs {

namespace {

constexpr int kThreads = 256;

struct BuildStats {
    int aabb[6];          // ordered-int min xyz, max xyz of kept means
    unsigned n_kept;
    unsigned n_invalid;
    unsigned hist[kSigmaBins];
    int sigma_grid_max;   // ordered-int max scale over the main tier
    unsigned n_main;      // kept Gaussians in the main tier
    unsigned dbg_err;     // kErrBounds: an index check of a CS_DEBUG build failed
};

__device__ __forceinline__ bool finite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Eq. 2 for one Gaussian: Sigma = (R S)(R S)^T with R from the (possibly
// unnormalised) quaternion via R = I - 2/|q|^2 (...) and S = diag(scale).
__global__ void __launch_bounds__(kThreads) k_repack(
    const float *__restrict__ means, const float *__restrict__ scales,
    const float *__restrict__ quats, const float *__restrict__ opacity, int64_t n, int use_filter,
    float opacity_min, float extent_max, float4 *__restrict__ pos, float4 *__restrict__ covA,
    float4 *__restrict__ covB, uint8_t *__restrict__ code, BuildStats *__restrict__ st) {
    __shared__ unsigned s_hist[kSigmaBins];
    __shared__ int s_box[6];
    __shared__ unsigned s_kept, s_bad;
    for (int b = threadIdx.x; b < kSigmaBins; b += kThreads) s_hist[b] = 0;
    if (threadIdx.x < 6) s_box[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
    if (threadIdx.x == 0) { s_kept = 0; s_bad = 0; }
    __syncthreads();

    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) {
        float mx = means[3 * i], my = means[3 * i + 1], mz = means[3 * i + 2];
        float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        float op = opacity ? opacity[i] : 1.f;
        bool ok = finite3(mx, my, mz) && finite3(s0, s1, s2) && finite3(qw, qx, qy) &&
                  isfinite(qz) && s0 >= 0.f && s1 >= 0.f && s2 >= 0.f && !isnan(op);
        float smax = fmaxf(fmaxf(s0, s1), s2);
        uint8_t c = 0;
        if (!ok) {
            c = 2;
            atomicAdd(&s_bad, 1u);
        } else if (use_filter && opacity && op < opacity_min && smax > extent_max) {
            c = 0;  // floater (Section II-C)
        } else {
            c = 1;
        }
        code[i] = c;
        if (c == 1) {
            float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
            if (!(n2 > 0.f)) { qw = 1.f; qx = qy = qz = 0.f; n2 = 1.f; }
            float s = 2.f / n2;
            float R00 = 1.f - s * (qy * qy + qz * qz), R01 = s * (qx * qy - qw * qz),
                  R02 = s * (qx * qz + qw * qy);
            float R10 = s * (qx * qy + qw * qz), R11 = 1.f - s * (qx * qx + qz * qz),
                  R12 = s * (qy * qz - qw * qx);
            float R20 = s * (qx * qz - qw * qy), R21 = s * (qy * qz + qw * qx),
                  R22 = 1.f - s * (qx * qx + qy * qy);
            // M = R diag(scale); Sigma = M M^T (a Gram matrix: PSD up to rounding)
            float M00 = R00 * s0, M01 = R01 * s1, M02 = R02 * s2;
            float M10 = R10 * s0, M11 = R11 * s1, M12 = R12 * s2;
            float M20 = R20 * s0, M21 = R21 * s1, M22 = R22 * s2;
            float Sxx = fmaf(M00, M00, fmaf(M01, M01, M02 * M02));
            float Syy = fmaf(M10, M10, fmaf(M11, M11, M12 * M12));
            float Szz = fmaf(M20, M20, fmaf(M21, M21, M22 * M22));
            float Sxy = fmaf(M00, M10, fmaf(M01, M11, M02 * M12));
            float Sxz = fmaf(M00, M20, fmaf(M01, M21, M02 * M22));
            float Syz = fmaf(M10, M20, fmaf(M11, M21, M12 * M22));
            pos[i] = make_float4(mx, my, mz, smax);
            covA[i] = make_float4(Sxx, Syy, Szz, 2.f * Sxy);
            covB[i] = make_float4(2.f * Sxz, 2.f * Syz, 0.f, __int_as_float((int)i));
            atomicAdd(&s_kept, 1u);
            int b = 0;
            if (smax > 0.f) {
                float l = (log2f(smax) - kSigmaLog2Lo) * kSigmaBinsPerOctave;
                b = (int)fminf(fmaxf(floorf(l), 0.f), (float)(kSigmaBins - 1));
            }
            atomicAdd(&s_hist[b], 1u);
            atomicMin(&s_box[0], float_to_ordered(mx));
            atomicMin(&s_box[1], float_to_ordered(my));
            atomicMin(&s_box[2], float_to_ordered(mz));
            atomicMax(&s_box[3], float_to_ordered(mx));
            atomicMax(&s_box[4], float_to_ordered(my));
            atomicMax(&s_box[5], float_to_ordered(mz));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSigmaBins; b += kThreads)
        if (s_hist[b]) atomicAdd(&st->hist[b], s_hist[b]);
    if (threadIdx.x < 3) atomicMin(&st->aabb[threadIdx.x], s_box[threadIdx.x]);
    else if (threadIdx.x < 6) atomicMax(&st->aabb[threadIdx.x], s_box[threadIdx.x]);
    if (threadIdx.x == 0) {
        if (s_kept) atomicAdd(&st->n_kept, s_kept);
        if (s_bad) atomicAdd(&st->n_invalid, s_bad);
    }
}

struct OrderParams {
    float lo[3];
    float inv_cube;     // 2^kSceneOrderBits / (edge of the scene cube)
    float sigma_tier;   // Gaussians with a larger max scale form the large tier
};

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3FFu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ uint32_t grid_coord(float x, float lo, float inv) {
    const float f = (x - lo) * inv;
    return (uint32_t)min(max((int)floorf(f), 0), (1 << kSceneOrderBits) - 1);
}

// Index of the cell (x, y, z) (10 bits per axis) along the 3-D Hilbert curve
// of 2^30 cells: J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc.
// 707 (2004).  The coordinates are turned into the curve's "transpose" form
// (undo the excess rotations level by level, then Gray-decode), whose bits,
// interleaved with x's bit first in each triple, are the index.  Consecutive
// indices are face-adjacent cells, so runs of consecutive Gaussians (the
// chunks) are more compact than along the Morton curve, which jumps at every
// octant boundary: about 6 % fewer (primitive, chunk) tests pass on the
// tabletop workloads.
__device__ __forceinline__ uint32_t hilbert3_10(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t X[3] = {x, y, z};
#pragma unroll
    for (uint32_t Q = 1u << (kSceneOrderBits - 1); Q > 1u; Q >>= 1) {
        const uint32_t P = Q - 1u;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;  // invert the low bits of x
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;  // exchange the low bits of x and axis i
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0u;
#pragma unroll
    for (uint32_t Q = 1u << (kSceneOrderBits - 1); Q > 1u; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1u;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    return (spread10(X[0]) << 2) | (spread10(X[1]) << 1) | spread10(X[2]);
}

// Sort key of each Gaussian: tier bit above the 30-bit Hilbert index of its
// mean; dropped rows sort last.
__global__ void __launch_bounds__(kThreads) k_keys(const float4 *__restrict__ pos,
                                                   const uint8_t *__restrict__ code, int64_t n,
                                                   OrderParams g, uint32_t *__restrict__ keys,
                                                   uint32_t *__restrict__ vals,
                                                   BuildStats *__restrict__ st) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i >= n) return;
    uint32_t key = 0xFFFFFFFFu;
    if (code[i] == 1) {
        const float4 p = pos[i];
        const uint32_t m = hilbert3_10(grid_coord(p.x, g.lo[0], g.inv_cube), grid_coord(p.y, g.lo[1], g.inv_cube),
                                       grid_coord(p.z, g.lo[2], g.inv_cube));
        const bool large = p.w > g.sigma_tier;
        key = (large ? 0x40000000u : 0u) | m;
        if (!large) {
            atomicMax(&st->sigma_grid_max, float_to_ordered(p.w));
            atomicAdd(&st->n_main, 1u);
        }
    }
    keys[i] = key;
    vals[i] = (uint32_t)i;
}

// Means in sorted order (input of the greedy chunking).
__global__ void k_gather_pos(const uint32_t *__restrict__ perm, const float4 *__restrict__ pos, int n,
                             float4 *__restrict__ spos, int n_in, unsigned *dbg) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n && CS_IDX_OK(perm[p] < (uint32_t)n_in, dbg)) spos[p] = pos[perm[p]];
}

// Greedy chunking, one thread per segment of kSegment sorted Gaussians
// (segments split the two tiers separately, and every segment starts a new
// chunk): a chunk takes the next Gaussian unless it already holds 32 or its
// box would exceed `extent` along an axis.  Without `base`, writes the
// segment's chunk count; with it (the exclusive scan of the counts), writes
// each Gaussian's slot = 32 * chunk + lane.
__global__ void k_chunk_greedy(const float4 *__restrict__ spos, int n_main, int n_kept, int seg_main,
                               int nseg, float ext_main, float ext_large, const uint32_t *__restrict__ base,
                               uint32_t *__restrict__ counts, uint32_t *__restrict__ slot, unsigned *dbg) {
    const int sg = blockIdx.x * blockDim.x + threadIdx.x;
    if (sg >= nseg) return;
    int p0, p1;
    if (sg < seg_main) {
        p0 = sg * kSegment;
        p1 = min(n_main, p0 + kSegment);
    } else {
        p0 = n_main + (sg - seg_main) * kSegment;
        p1 = min(n_kept, p0 + kSegment);
    }
    const float L = sg < seg_main ? ext_main : ext_large;
    const uint32_t c0 = base ? base[sg] : 0u;
    uint32_t c = 0;
    int k = 0;
    float lx = 0.f, ly = 0.f, lz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    for (int p8 = p0; p8 < p1; p8 += 8) {
        float4 P8[8];  // the next eight means in flight at once
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (p8 + u < p1) P8[u] = spos[p8 + u];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int p = p8 + u;
            if (p >= p1) break;
            const float4 P = P8[u];
            if (k > 0) {
                const float nlx = fminf(lx, P.x), nly = fminf(ly, P.y), nlz = fminf(lz, P.z);
                const float nhx = fmaxf(hx, P.x), nhy = fmaxf(hy, P.y), nhz = fmaxf(hz, P.z);
                if (k == kChunk || fmaxf(fmaxf(nhx - nlx, nhy - nly), nhz - nlz) > L) {
                    ++c;
                    k = 0;
                } else {
                    lx = nlx; ly = nly; lz = nlz; hx = nhx; hy = nhy; hz = nhz;
                }
            }
            if (k == 0) {
                lx = hx = P.x; ly = hy = P.y; lz = hz = P.z;
            }
            // base[nseg] is the chunk count: every slot must lie below 32 times it
            if (base && CS_IDX_OK(c0 + c < base[nseg], dbg)) slot[p] = (c0 + c) * kChunk + (uint32_t)k;
            ++k;
        }
    }
    if (!base) counts[sg] = p1 > p0 ? c + 1 : 0u;
}

// Every slot starts as padding: a point at 1e18 with zero covariance.
__global__ void k_fill_padding(ChunkBlock *__restrict__ blocks, int nchunks, float *__restrict__ slot_smax) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nchunks * kChunk) return;
    ChunkBlock &b = blocks[t / kChunk];
    int l = t % kChunk;
    b.x[l] = 1e18f; b.y[l] = 1e18f; b.z[l] = 1e18f;
    b.sxx[l] = 0.f; b.syy[l] = 0.f; b.szz[l] = 0.f;
    b.sxy2[l] = 0.f; b.sxz2[l] = 0.f; b.syz2[l] = 0.f;
    slot_smax[t] = -1.f;  // marks padding for the header pass
}

// Sorted Gaussian p goes to slot[p].
__global__ void k_scatter_slots(const uint32_t *__restrict__ slot_in, const uint32_t *__restrict__ perm,
                                int n_gauss, const float4 *__restrict__ pos, const float4 *__restrict__ covA,
                                const float4 *__restrict__ covB, ChunkBlock *__restrict__ blocks,
                                float *__restrict__ slot_smax, float *__restrict__ smax,
                                int32_t *__restrict__ index, int32_t *__restrict__ slot_of, int nchunks,
                                int n_in, unsigned *dbg) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_gauss) return;
    const uint32_t slot = slot_in[p];
    const uint32_t i = perm[p];
    if (!CS_IDX_OK(slot < (uint32_t)nchunks * kChunk && i < (uint32_t)n_in, dbg)) return;
    const float4 P = pos[i], A = covA[i], B = covB[i];
    ChunkBlock &b = blocks[slot / kChunk];
    const int l = (int)(slot % kChunk);
    b.x[l] = P.x; b.y[l] = P.y; b.z[l] = P.z;
    b.sxx[l] = A.x; b.syy[l] = A.y; b.szz[l] = A.z; b.sxy2[l] = A.w;
    b.sxz2[l] = B.x; b.syz2[l] = B.y;
    slot_smax[slot] = P.w;
    smax[p] = P.w;
    index[p] = (int32_t)i;
    slot_of[p] = (int32_t)slot;
}

// One warp per chunk: the box of its real slots, their largest scale and
// their number, into the block header and the compact chunk-box array.
__global__ void k_chunk_headers(ChunkBlock *__restrict__ blocks, int nchunks, const float *__restrict__ slot_smax,
                                NodeBox *__restrict__ chead) {
    int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (c >= nchunks) return;
    ChunkBlock &b = blocks[c];
    const float sg0 = slot_smax[(size_t)c * kChunk + lane];
    const bool real = sg0 >= 0.f;
    float lx = real ? b.x[lane] : INFINITY, ly = real ? b.y[lane] : INFINITY, lz = real ? b.z[lane] : INFINITY;
    float hx = real ? b.x[lane] : -INFINITY, hy = real ? b.y[lane] : -INFINITY, hz = real ? b.z[lane] : -INFINITY;
    float sg = real ? sg0 : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        sg = fmaxf(sg, __shfl_xor_sync(0xffffffffu, sg, o));
    }
    const int nreal = __popc(__ballot_sync(0xffffffffu, real));
    if (lane == 0) {
        const float4 lo = make_float4(lx, ly, lz, sg), hi = make_float4(hx, hy, hz, (float)nreal);
        b.lo = lo;
        b.hi = hi;
        chead[c] = NodeBox{lo, hi};
    }
}

// One warp per node: the union of its (up to) 32 children.
__global__ void k_node_level(const NodeBox *__restrict__ child, int nchild, NodeBox *__restrict__ node, int nnode) {
    int k = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    int lane = threadIdx.x & 31;
    if (k >= nnode) return;
    const int c = k * 32 + lane;
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY, sg = 0.f;
    if (c < nchild) {
        const NodeBox b = child[c];
        lx = b.lo.x; ly = b.lo.y; lz = b.lo.z; sg = b.lo.w;
        hx = b.hi.x; hy = b.hi.y; hz = b.hi.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
        sg = fmaxf(sg, __shfl_xor_sync(0xffffffffu, sg, o));
    }
    if (lane == 0) node[k] = NodeBox{make_float4(lx, ly, lz, sg), make_float4(hx, hy, hz, 0.f)};
}

// A temporary of the build, allocated from the library's stream-ordered pool
// on the build's stream and returned to it in stream order (no cudaFree, so
// no device-wide synchronisation per temporary).
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
};

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

cudaError_t temp_alloc(DevBuf &b, cudaStream_t s, size_t bytes) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = temp_pool(&pool);
    if (e != cudaSuccess) return e;
    b.s = s;
    return cudaMallocFromPoolAsync(&b.p, bytes, pool, s);
}

}  // namespace

cs_status build_scene(const cs_scene_desc *d, cudaStream_t s, Scene *sc) {
    const int64_t n = d->n;
    sc->n_input = n;
    DevBuf in_means, in_scales, in_quats, in_op, tmp_rec, tmp_code, tmp_kv, tmp_hist, tmp_scan,
        d_stats;
    const float *means = d->means, *scales = d->scales, *quats = d->quats, *op = d->opacity;
    if (n > 0 && !d->on_device) {
        CS_CUDA(temp_alloc(in_means, s, 12 * n));
        CS_CUDA(temp_alloc(in_scales, s, 12 * n));
        CS_CUDA(temp_alloc(in_quats, s, 16 * n));
        CS_CUDA(cudaMemcpyAsync(in_means.p, d->means, 12 * n, cudaMemcpyHostToDevice, s));
        CS_CUDA(cudaMemcpyAsync(in_scales.p, d->scales, 12 * n, cudaMemcpyHostToDevice, s));
        CS_CUDA(cudaMemcpyAsync(in_quats.p, d->quats, 16 * n, cudaMemcpyHostToDevice, s));
        means = (const float *)in_means.p;
        scales = (const float *)in_scales.p;
        quats = (const float *)in_quats.p;
        if (op) {
            CS_CUDA(temp_alloc(in_op, s, 4 * n));
            CS_CUDA(cudaMemcpyAsync(in_op.p, d->opacity, 4 * n, cudaMemcpyHostToDevice, s));
            op = (const float *)in_op.p;
        }
    }
    const int64_t nn = n > 0 ? n : 1;
    CS_CUDA(temp_alloc(tmp_rec, s, 48 * nn));
    CS_CUDA(temp_alloc(tmp_code, s, nn));
    CS_CUDA(temp_alloc(tmp_kv, s, 16 * nn));
    CS_CUDA(temp_alloc(d_stats, s, sizeof(BuildStats)));
    float4 *upos = (float4 *)tmp_rec.p, *ucovA = upos + nn, *ucovB = ucovA + nn;
    uint8_t *code = (uint8_t *)tmp_code.p;
    BuildStats hs;
    memset(&hs, 0, sizeof(hs));
    for (int k = 0; k < 3; ++k) { hs.aabb[k] = INT_MAX; hs.aabb[3 + k] = INT_MIN; }
    hs.sigma_grid_max = INT_MIN;
    CS_CUDA(cudaMemcpyAsync(d_stats.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    BuildStats *st = (BuildStats *)d_stats.p;
    if (n > 0) {
        k_repack<<<blocks_for(n), kThreads, 0, s>>>(means, scales, quats, op, n, d->use_filter,
                                                    d->opacity_min, d->extent_max, upos, ucovA,
                                                    ucovB, code, st);
        count_launches(1);
    }
    CS_CUDA(cudaGetLastError());
    CS_CUDA(cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    sc->n_invalid = hs.n_invalid;
    const int64_t kept_est = hs.n_kept;

    // ---- order parameters (host): extent of the kept means, tier cut, chunk extent
    float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    if (kept_est > 0) {
        for (int k = 0; k < 3; ++k) {
            int a = hs.aabb[k], b = hs.aabb[3 + k];
            lo[k] = __builtin_bit_cast(float, a >= 0 ? a : a ^ 0x7FFFFFFF);
            hi[k] = __builtin_bit_cast(float, b >= 0 ? b : b ^ 0x7FFFFFFF);
        }
    }
    float ext[3], emax = 0.f;
    for (int k = 0; k < 3; ++k) { ext[k] = hi[k] - lo[k]; emax = std::max(emax, ext[k]); }
    if (!(emax > 0.f)) emax = 1.f;
    const float ext_min = emax * 1e-3f;
    for (int k = 0; k < 3; ++k) ext[k] = std::max(ext[k], ext_min);
    // tier cut: the tier_quantile of the largest scale (upper edge of its bin)
    double q = d->tier_quantile > 0.f ? std::min(1.0, (double)d->tier_quantile) : 0.99;
    float sigma_tier = INFINITY;
    if (kept_est > 0 && q < 1.0) {
        uint64_t target = (uint64_t)ceil(q * (double)kept_est), cum = 0;
        for (int b = 0; b < kSigmaBins; ++b) {
            cum += hs.hist[b];
            if (cum >= target) {
                sigma_tier = exp2f(kSigmaLog2Lo + (float)(b + 1) / kSigmaBinsPerOctave);
                break;
            }
        }
    }
    // chunk extent limit: twice the edge of a box that holds 32 Gaussians at
    // the mean density of the bounding box (cell_size overrides); the large
    // tier, sparse by construction, allows four times that
    float h = d->cell_size;
    if (!(h > 0.f)) {
        double vol = (double)ext[0] * ext[1] * ext[2];
        h = 2.f * (float)cbrt(vol * 32.0 / (double)std::max<int64_t>(kept_est, 1));
    }
    h = std::max(h, emax / 1024.f);
    OrderParams g;
    for (int k = 0; k < 3; ++k) g.lo[k] = lo[k];
    g.inv_cube = (float)(1 << kSceneOrderBits) / emax;
    g.sigma_tier = sigma_tier;

    // ---- keys, stable sort
    uint32_t *keys[2] = {(uint32_t *)tmp_kv.p, (uint32_t *)tmp_kv.p + nn};
    uint32_t *vals[2] = {(uint32_t *)tmp_kv.p + 2 * nn, (uint32_t *)tmp_kv.p + 3 * nn};
    size_t hist_n = sort_hist_elems((size_t)nn);
    const int64_t nseg_max = 2 + (nn + kSegment - 1) / kSegment;
    size_t scan_n = scan_tmp_elems(std::max(hist_n, (size_t)nseg_max + 1));
    CS_CUDA(temp_alloc(tmp_hist, s, 4 * std::max(hist_n, (size_t)nseg_max + 1)));
    CS_CUDA(temp_alloc(tmp_scan, s, 4 * scan_n));
    int res = 0;
    if (n > 0) {
        k_keys<<<blocks_for(n), kThreads, 0, s>>>(upos, code, n, g, keys[0], vals[0], st);
        count_launches(1);
        res = radix_sort(keys, vals, (size_t)n, 32, (uint32_t *)tmp_hist.p, (uint32_t *)tmp_scan.p, s);
    }
    unsigned n_main_u = 0;
    int sgm = INT_MIN;
    CS_CUDA(cudaMemcpyAsync(&n_main_u, &st->n_main, 4, cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaMemcpyAsync(&sgm, &st->sigma_grid_max, 4, cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaStreamSynchronize(s));
    const int64_t n_kept = kept_est, n_main = n_main_u;
    if (n_kept > ((int64_t)1 << 31) / 2) {
        set_error("scene too large (more than 2^30 kept Gaussians)");
        return CS_ERR_INVALID_ARG;
    }

    // ---- greedy chunking in segments, then chunk bases by a scan
    const int seg_main = (int)((n_main + kSegment - 1) / kSegment);
    const int nseg = seg_main + (int)((n_kept - n_main + kSegment - 1) / kSegment);
    DevBuf tmp_spos, tmp_cnt, tmp_base, tmp_slot;
    CS_CUDA(temp_alloc(tmp_spos, s, 16 * (size_t)std::max<int64_t>(n_kept, 1)));
    CS_CUDA(temp_alloc(tmp_cnt, s, 4 * ((size_t)nseg + 1)));
    CS_CUDA(temp_alloc(tmp_base, s, 4 * ((size_t)nseg + 1)));
    CS_CUDA(temp_alloc(tmp_slot, s, 4 * (size_t)std::max<int64_t>(n_kept, 1)));
    float4 *spos = (float4 *)tmp_spos.p;
    uint32_t *seg_cnt = (uint32_t *)tmp_cnt.p, *seg_base = (uint32_t *)tmp_base.p, *slot = (uint32_t *)tmp_slot.p;
    const float ext_main = h, ext_large = 4.f * h;
    CS_CUDA(cudaMemsetAsync(seg_cnt, 0, 4 * ((size_t)nseg + 1), s));
    if (n_kept > 0) {
        k_gather_pos<<<blocks_for(n_kept), kThreads, 0, s>>>(vals[res], upos, (int)n_kept, spos, (int)n,
                                                             &st->dbg_err);
        k_chunk_greedy<<<(nseg + 127) / 128, 128, 0, s>>>(spos, (int)n_main, (int)n_kept, seg_main, nseg, ext_main,
                                                          ext_large, nullptr, seg_cnt, nullptr, &st->dbg_err);
        count_launches(2);
    }
    scan_exclusive(seg_cnt, seg_base, (size_t)nseg + 1, (uint32_t *)tmp_scan.p, s);
    uint32_t bounds[2] = {0, 0};  // first chunk of the large tier, number of chunks
    CS_CUDA(cudaMemcpyAsync(&bounds[0], seg_base + seg_main, 4, cudaMemcpyDeviceToHost, s));
    CS_CUDA(cudaMemcpyAsync(&bounds[1], seg_base + nseg, 4, cudaMemcpyDeviceToHost, s));
    if (n_kept > 0) {
        k_chunk_greedy<<<(nseg + 127) / 128, 128, 0, s>>>(spos, (int)n_main, (int)n_kept, seg_main, nseg, ext_main,
                                                          ext_large, seg_base, nullptr, slot, &st->dbg_err);
        count_launches(1);
    }
    CS_CUDA(cudaGetLastError());
    CS_CUDA(cudaStreamSynchronize(s));
    const int nchunks = (int)bounds[1];
    if (nchunks > ((int64_t)1 << 31) / kChunk) {
        set_error("internal: chunk count overflow in scene build");
        return CS_ERR_CUDA;
    }
    int nnodes[kLevels];
    {
        int m = nchunks;
        for (int l = 0; l < kLevels; ++l) {
            m = (m + 31) / 32;
            nnodes[l] = std::max(m, nchunks > 0 ? 1 : 0);
        }
    }

    // owned memory: chunk blocks, chunk boxes, node levels, and per sorted
    // Gaussian its largest scale, input row and slot (export)
    const int64_t kmax = std::max<int64_t>(n_kept, 1);
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = align(sizeof(ChunkBlock) * (size_t)std::max(nchunks, 1));
    const size_t off_chead = off;
    off = align(off + sizeof(NodeBox) * (size_t)std::max(nchunks, 1));
    size_t off_nodes[kLevels];
    for (int l = 0; l < kLevels; ++l) {
        off_nodes[l] = off;
        off = align(off + sizeof(NodeBox) * (size_t)std::max(nnodes[l], 1));
    }
    const size_t off_smax = off;
    const size_t off_index = align(off_smax + 4 * (size_t)kmax);
    const size_t off_slot = align(off_index + 4 * (size_t)kmax);
    const size_t total = off_slot + 4 * (size_t)kmax;
    void *blk = nullptr;
    cudaError_t e = cudaMalloc(&blk, total);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation
                                     ? (set_error("scene allocation failed"), CS_ERR_NO_MEMORY)
                                     : cuda_fail(e, "cudaMalloc(scene)");
    sc->blocks[sc->nblocks++] = blk;
    sc->device_bytes = (int64_t)total;
    char *base = (char *)blk;
    ChunkBlock *blocks = (ChunkBlock *)base;
    NodeBox *chead = (NodeBox *)(base + off_chead);
    NodeBox *nodes[kLevels];
    for (int l = 0; l < kLevels; ++l) nodes[l] = (NodeBox *)(base + off_nodes[l]);
    float *smax = (float *)(base + off_smax);
    int32_t *index = (int32_t *)(base + off_index);
    int32_t *slot_of = (int32_t *)(base + off_slot);
    if (nchunks > 0) {
        DevBuf tmp_ss;
        CS_CUDA(temp_alloc(tmp_ss, s, 4 * (size_t)nchunks * kChunk));
        float *slot_smax = (float *)tmp_ss.p;
        k_fill_padding<<<(unsigned)(((int64_t)nchunks * kChunk + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            blocks, nchunks, slot_smax);
        k_scatter_slots<<<blocks_for(n_kept), kThreads, 0, s>>>(slot, vals[res], (int)n_kept, upos, ucovA, ucovB,
                                                                blocks, slot_smax, smax, index, slot_of, nchunks,
                                                                (int)n, &st->dbg_err);
        k_chunk_headers<<<(unsigned)(((int64_t)nchunks * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            blocks, nchunks, slot_smax, chead);
        count_launches(3);
        const NodeBox *child = chead;
        int nchild = nchunks;
        for (int l = 0; l < kLevels; ++l) {
            k_node_level<<<(unsigned)(((int64_t)nnodes[l] * 32 + kThreads - 1) / kThreads), kThreads, 0, s>>>(
                child, nchild, nodes[l], nnodes[l]);
            count_launches(1);
            child = nodes[l];
            nchild = nnodes[l];
        }
        CS_CUDA(cudaGetLastError());
    }
    CS_CUDA(cudaGetLastError());
    CS_CUDA(cudaStreamSynchronize(s));  // the scene is complete when cs_scene_create returns
    if (kDebugBuild) {
        unsigned dbg = 0;
        CS_CUDA(cudaMemcpy(&dbg, &st->dbg_err, sizeof(dbg), cudaMemcpyDeviceToHost));
        if (dbg) {
            set_error("a device-side index check failed in the scene build (CS_DEBUG build)");
            return CS_ERR_BOUNDS;
        }
    }

    sc->n_kept = n_kept;
    sc->n_grid = n_main;
    sc->n_large = n_kept - n_main;
    SceneDev &dv = sc->dev;
    dv.blocks = blocks;
    dv.chead = chead;
    for (int l = 0; l < kLevels; ++l) {
        dv.nodes[l] = nodes[l];
        dv.nnodes[l] = nchunks > 0 ? nnodes[l] : 0;
    }
    dv.smax = smax;
    dv.index = index;
    dv.slot_of = slot_of;
    dv.n_gauss = (int)n_kept;
    dv.nchunks = nchunks;
    dv.large_chunk0 = (int)bounds[0];
    dv.chunk_extent = ext_main;
    for (int k = 0; k < 3; ++k) {
        dv.bb_lo[k] = lo[k];
        dv.bb_hi[k] = lo[k] + ext[k];
    }
    float sg = 0.f;
    if (sgm != INT_MIN) sg = __builtin_bit_cast(float, sgm >= 0 ? sgm : sgm ^ 0x7FFFFFFF);
    dv.sigma_tier = sg;
    // slack for the FP32 rounding of distances and box gaps
    float amax = 0.f;
    for (int k = 0; k < 3; ++k) amax = std::max({amax, fabsf(lo[k]), fabsf(hi[k])});
    dv.pad_abs = 4e-6f * std::max(amax, emax) + 1e-30f;
    return CS_OK;
}

namespace {
// Unpack the chunk blocks into row-major arrays (cs_scene_export).
__global__ void k_export(const ChunkBlock *__restrict__ blocks, const float *__restrict__ smax,
                         const int32_t *__restrict__ index, const int32_t *__restrict__ slot_of, int n,
                         float *__restrict__ pos, float *__restrict__ cov, int32_t *__restrict__ oidx) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int t = slot_of[p];
    const ChunkBlock &b = blocks[t / kChunk];
    int l = t % kChunk;
    if (pos) {
        pos[4 * p + 0] = b.x[l]; pos[4 * p + 1] = b.y[l]; pos[4 * p + 2] = b.z[l];
        pos[4 * p + 3] = smax[p];
    }
    if (cov) {
        float *c = cov + 8 * (size_t)p;
        c[0] = b.sxx[l]; c[1] = b.syy[l]; c[2] = b.szz[l];
        c[3] = b.sxy2[l]; c[4] = b.sxz2[l]; c[5] = b.syz2[l];
        c[6] = 0.f; c[7] = 0.f;
    }
    if (oidx) oidx[p] = index[p];
}
}  // namespace

void launch_export(const SceneDev &sc, float *pos, float *cov, int32_t *index, cudaStream_t s) {
    k_export<<<(sc.n_gauss + 255) / 256, 256, 0, s>>>(sc.blocks, sc.smax, sc.index, sc.slot_of, sc.n_gauss, pos,
                                                      cov, index);
    count_launches(1);
}

}  // namespace cs
