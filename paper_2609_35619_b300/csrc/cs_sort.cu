// cs_sort.cu -- device-wide exclusive scan and stable LSD radix sort used to
// build the uniform grid over the Gaussians and to order queries spatially.
#include "cs_internal.cuh"

namespace cs {

// ------------------------------------------------------------------- scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024 elements per block

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive block scan of one value per thread.
__device__ __forceinline__ void block_excl_scan(uint32_t v, uint32_t &excl) {
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v, lane);
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        uint32_t ti = warp_incl_scan(t, lane);
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;  // exclusive
    }
    __syncthreads();
    excl = incl - v + warp_tot[w];
}

__global__ void k_scan_sums(const uint32_t *__restrict__ in, size_t n, uint32_t *__restrict__ sums) {
    size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + (size_t)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    // block reduction
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t red[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void k_scan_apply(const uint32_t *__restrict__ in, uint32_t *__restrict__ out, size_t n,
                             const uint32_t *__restrict__ block_offsets) {
    size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + (size_t)threadIdx.x * kScanItems + k;
        v[k] = i < n ? in[i] : 0u;
        local += v[k];
    }
    uint32_t excl;
    block_excl_scan(local, excl);
    uint32_t run = excl + (block_offsets ? block_offsets[blockIdx.x] : 0u);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + (size_t)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
}

size_t scan_tmp_elems(size_t n) {
    size_t total = 0;
    while (n > (size_t)kScanTile) {
        size_t nb = (n + kScanTile - 1) / kScanTile;
        total += nb;
        n = nb;
    }
    return total + 1;
}

void scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s) {
    if (n == 0) return;
    size_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_apply<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        count_launches(1);
        return;
    }
    uint32_t *sums = tmp;
    k_scan_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    scan_exclusive(sums, sums, nb, tmp + nb, s);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
    count_launches(2);
}

// ------------------------------------------------------------- radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 4096 elements per block
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(const uint32_t *__restrict__ keys,
                                                            size_t n, int shift,
                                                            uint32_t *__restrict__ hist,
                                                            unsigned nblocks) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        size_t i = base + (size_t)r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xFFu], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: items are ranked in index order (round, warp, lane).
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, size_t n, int shift, const uint32_t *__restrict__ offsets,
    unsigned nblocks) {
    __shared__ uint32_t run[kRadix];
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    run[threadIdx.x] = offsets[(size_t)threadIdx.x * nblocks + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    size_t base = (size_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortRounds; ++r) {
        size_t r0 = base + (size_t)r * kSortThreads;
        if (r0 >= n) break;  // uniform across the block
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) wcnt[k][threadIdx.x] = 0;
        __syncthreads();
        size_t i = r0 + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? kin[i] : 0u;
        uint32_t val = valid ? vin[i] : 0u;
        int d = valid ? (int)((key >> shift) & 0xFFu) : kRadix;  // invalid lanes form their own group
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0;
            for (int k = 0; k < w; ++k) pre += wcnt[k][d];
            uint32_t pos = run[d] + pre + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) tot += wcnt[k][threadIdx.x];
        run[threadIdx.x] += tot;
        __syncthreads();
    }
}

size_t sort_hist_elems(size_t n) {
    size_t nb = (n + kSortTile - 1) / kSortTile;
    return (size_t)kRadix * (nb > 0 ? nb : 1);
}

int radix_sort(uint32_t *keys[2], uint32_t *vals[2], size_t n, int bits, uint32_t *hist,
               uint32_t *scan_tmp, cudaStream_t s) {
    int cur = 0;
    if (n <= 1) return cur;
    unsigned nb = (unsigned)((n + kSortTile - 1) / kSortTile);
    for (int shift = 0; shift < bits; shift += 8) {
        k_sort_hist<<<nb, kSortThreads, 0, s>>>(keys[cur], n, shift, hist, nb);
        scan_exclusive(hist, hist, (size_t)kRadix * nb, scan_tmp, s);
        k_sort_scatter<<<nb, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                   vals[cur ^ 1], n, shift, hist, nb);
        count_launches(2);
        cur ^= 1;
    }
    return cur;
}

}  // namespace cs
