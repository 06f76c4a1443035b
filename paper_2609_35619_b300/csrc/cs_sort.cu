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

// Stable scatter.  Warp w of a block owns keys [w 512, (w + 1) 512) of the
// block's 4,096 (16 rounds of 32 in index order).  Pass 1 counts each warp's
// digits; the counts then give every digit its start in the block and every
// warp its first slot per digit; pass 2 places each warp's keys in index
// order (lanes of equal digit ranked by lane) into shared memory, sorted by
// digit; a last pass writes each digit's run to its place in the output
// (the block's offset from the global scan), so stores are contiguous runs
// instead of one scattered 4-byte write per key.  Equal digits keep their
// index order: the sort is stable.
__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(
    const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin, uint32_t *__restrict__ kout,
    uint32_t *__restrict__ vout, size_t n, int shift, const uint32_t *__restrict__ offsets,
    unsigned nblocks) {
    constexpr int kPerWarp = kSortTile / kSortWarps;  // 512
    __shared__ uint32_t cnt[kSortWarps][kRadix];
    __shared__ uint32_t lstart[kRadix], goff[kRadix];
    __shared__ uint32_t skey[kSortTile], sval[kSortTile];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const size_t tile0 = (size_t)blockIdx.x * kSortTile;
    const size_t base = tile0 + (size_t)w * kPerWarp;
    for (int d = lane; d < kRadix; d += 32) cnt[w][d] = 0;
    __syncwarp();
    for (int r = 0; r < kPerWarp / 32; ++r) {
        const size_t i = base + (size_t)r * 32 + lane;
        const bool valid = i < n;
        const int d = valid ? (int)((kin[i] >> shift) & 0xFFu) : kRadix;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && (peers & lt_mask) == 0u) cnt[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // one thread per digit
        uint32_t tot = 0;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) tot += cnt[k][d];
        uint32_t start;
        block_excl_scan(tot, start);  // the digit's first slot in the block
        lstart[d] = start;
        goff[d] = offsets[(size_t)d * nblocks + blockIdx.x];
        uint32_t run = start;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) {
            const uint32_t c = cnt[k][d];
            cnt[k][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < kPerWarp / 32; ++r) {
        const size_t i = base + (size_t)r * 32 + lane;
        const bool valid = i < n;
        const uint32_t key = valid ? kin[i] : 0u;
        const uint32_t val = valid ? vin[i] : 0u;
        const int d = valid ? (int)((key >> shift) & 0xFFu) : kRadix;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const unsigned rank = __popc(peers & lt_mask);
        const uint32_t lp = valid ? cnt[w][d] + rank : 0u;
        __syncwarp();
        if (valid && rank == 0u) cnt[w][d] += __popc(peers);
        __syncwarp();
        if (valid) {
            skey[lp] = key;
            sval[lp] = val;
        }
    }
    __syncthreads();
    const int tn = (int)min((size_t)kSortTile, n - tile0);
    for (int lp = threadIdx.x; lp < tn; lp += kSortThreads) {
        const uint32_t key = skey[lp];
        const int d = (int)((key >> shift) & 0xFFu);
        const uint32_t pos = goff[d] + (uint32_t)lp - lstart[d];
        kout[pos] = key;
        vout[pos] = sval[lp];
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
