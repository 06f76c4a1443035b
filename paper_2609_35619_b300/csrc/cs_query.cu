// cs_query.cu -- the query path: spatial ordering of the primitives, the
// fused cull + pair evaluation + per-primitive reduction kernel (forward and
// adjoint), and the group epilogue.
//
// Fused kernel layout (one CTA per tile of TQ consecutive sorted primitives):
//   warp NCW        producer: computes the tile's bounding box and reach,
//                   descends the chunk tree to the chunks within reach (the
//                   cull), stages each run of them into a ring of NS
//                   shared-memory stages with one 1-D bulk copy completing on
//                   the stage's mbarrier, and while the copy flies tests every
//                   staged chunk against every primitive of the tile (lane =
//                   primitive, one ballot per 32), leaving a hit mask per slot;
//   warps 0..NCW-1  consumers: each owns QW primitives; per stage it takes the
//                   slots its bits of the hit masks mark, lane l evaluating
//                   slot l of a chunk (two chunks at once in packed FP32x2 for
//                   sphere cost reductions) against the primitives that reach
//                   it, with per-lane reductions reduced across lanes at the
//                   end by fixed shuffle trees.
#include <float.h>
#include <math.h>

#include <algorithm>
#include <atomic>

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
    int exact;      // sigma^2 is the exact variance of the quadratic form (Eq. 5)
    int sweep;      // n_sigma blocks of a conservatism sweep (1: none)
    // The packed cost path leaves out the clamp max(., 0) of Eq. 8.  A
    // negative unclamped st2 must then give what the clamped 0 gives:
    float S_cut_u;  // S_cut, or -inf when S_cut < 0 (then 0 is no neighbour)
    float T_in_u;   // T_in, or -inf when T_in <= 0
    float E_cap;    // min(G s_min, 0), the cap of the Eq. 11 exponent
};

struct EvalArgs {
    SceneDev sc;
    const float4 *qrec;      // prepared primitives, sorted order, RECS float4 each
    const float *qns;        // n_sigma per sorted primitive (not read by sweeps)
    const uint32_t *perm;    // sorted position -> input row
    int Q;                   // launch rows (S Qb for a sweep)
    // A conservatism sweep (S > 1) evaluates S copies of each of the Qb
    // prepared primitives: launch row q = p S + s is sorted primitive p at
    // n_sigma sw.v[s], written to output row s Qb + perm[p].  The copies are
    // made here, row by row, so no expanded records exist in memory.
    int S;
    int Qb;
    SweepNs sw;
    // persistent shapes: tiles are taken from this per-launch counter (zeroed
    // before the launch), ntiles of them
    int *tile_ctr;
    int ntiles;
    int num_sms;
    QueryConsts k;
    float *out_metric;
    uint8_t *out_collide;
    int32_t *out_count;
    const float *grad_out;   // GRAD: upstream per row (or per group)
    float *grad_centres;     // GRAD: [Q,3]
    unsigned *err;
    unsigned long long *stats;
    unsigned long long *kstats;  // optional kernel counters (see cs_params.out_kernel_stats)
    long long wait_polls;
    unsigned *gflags;        // flags mode with groups: per group, set once a row of it collides
};

// Launch row q: its prepared record, its n_sigma and its output row.
template <int RECS>
__device__ __forceinline__ const float4 *row_rec(const EvalArgs &a, int q) {
    const int p = a.S > 1 ? q / a.S : q;
    return a.qrec + (size_t)(CS_IDX_OK(p >= 0 && p < a.Qb, a.err) ? p : 0) * RECS;
}
__device__ __forceinline__ float row_ns(const EvalArgs &a, int q) {
    return a.S > 1 ? a.sw.v[q % a.S] : a.qns[q];
}
__device__ __forceinline__ uint32_t row_out(const EvalArgs &a, int q) {
    uint32_t r;
    if (a.S > 1) {
        const int p = q / a.S;
        r = (uint32_t)(q - p * a.S) * (uint32_t)a.Qb + a.perm[p];
    } else {
        r = a.perm[q];
    }
    // an output row outside the launch's rows would be written out of range:
    // a CS_DEBUG build records it and redirects the write to row 0
    return CS_IDX_OK(r < (uint32_t)a.Q, a.err) ? r : 0u;
}

// Kernel shape: NCW consumer warps, each owning QW primitives of the tile,
// one producer warp, NS pipeline stages of CHB chunk blocks each, and MINB
// CTAs resident per SM (the register budget follows from it).
// GROUP (packed sphere-cost path): primitives are evaluated in groups of
// GROUP whenever any member reaches the chunk (a member that does not adds
// exactly nothing, st2 > S_cut); larger groups give the scheduler more
// independent dependency chains per basic block.  GROUP == QW drops the
// per-primitive test altogether.
template <int NCW_, int QW_, int NS_, int CHB_, int MINB_, int GROUP_ = 2, int IL_ = 0, bool PERSIST_ = false>
struct Cfg {
    static constexpr int NCW = NCW_, QW = QW_, NS = NS_, CHB = CHB_, MINB = MINB_, GROUP = GROUP_;
    // PERSIST: a grid of (SMs x MINB) CTAs, each taking tiles from a device
    // counter until none are left; the producer warp culls and stages the next
    // tile while the consumer warps finish the current one (the stage ring runs
    // on across tiles, a terminator stage between them)
    static constexpr bool PERSIST = PERSIST_;
    // IL = 0: consumer warp w takes rows w QW .. w QW + QW - 1 of the tile (a
    // compact warp box); IL = 1: rows w, w + NCW, ...; IL = 2: row pairs
    // (2w, 2w + 1), (2w + 2 NCW, 2w + 2 NCW + 1), ...; IL = 4: row quads
    // (4w .. 4w + 3), (4w + 4 NCW ..), ...  Spreading a warp's primitives
    // over the tile evens out the warps' loads (they share the stage ring, so
    // the slowest sets the pace); pairs and quads keep the primitives
    // evaluated together close (the four n_sigma copies of a sweep).
    static constexpr int IL = IL_;
    __device__ static int row(int warp, int j) {
        return IL == 1 ? j * NCW + warp
             : IL == 2 ? (j >> 1) * 2 * NCW + 2 * warp + (j & 1)
             : IL == 4 ? (j >> 2) * 4 * NCW + 4 * warp + (j & 3)
                       : warp * QW + j;
    }
    static_assert(CHB <= 32, "one lane tests each chunk slot of a stage");
    static_assert(QW == 8 || QW == 16, "primitive masks are tested 32 / QW chunks per round");
    static_assert(IL == 0 || IL == 1 || IL == 2 || IL == 4, "row layouts");
    // warp rows j and j + 2 (j even) are consecutive tile rows: a sweep's
    // copies can share their geometry over four rows, not just two
    static constexpr bool QUAD = IL == 0 || IL == 4;
};

struct SlotMeta {
    int chunk;  // global chunk id
    int lo;     // 0
    int hi;     // real slots of the chunk (0: no chunk)
    int pad;
};

// Variants of the sphere cost kernels (the SH template parameter, bit flags):
// kShGeom: the n_sigma copies of a conservatism sweep share their pair
// geometry; kShK0: k_thr = 0, so a row collides iff its smallest st2 is
// below T_in, and a running minimum replaces the in-collision count.
constexpr int kShGeom = 1;
constexpr int kShK0 = 2;
// kShFwd (adjoint launches, spheres, cost modes): the same launch also writes
// the forward outputs (metric, flag, count) from the pairs it evaluates.
constexpr int kShFwd = 4;
// kShQuad (with kShGeom, on the row-quad shapes that evaluate groups of four):
// the sweep has a multiple of four n_sigma values, so every row quad of a
// tile is four copies of one prepared sphere (launch rows 4m .. 4m + 3 are
// p S + s .. p S + s + 3), or four dead rows (beyond the batch, or a sphere
// whose record is invalid).  Only the quad evaluation is compiled: no
// per-row fallback, fewer registers.  A dead quad's record has live = 0,
// so its reach test never passes and it is never evaluated.
constexpr int kShQuad = 8;

// Per-primitive data in shared memory, 4 float4 (QREC) per primitive:
//   sphere:    (c, 1/r^2) (2n, alpha, beta, live) - -
//   ellipsoid: (c, 2n) (Axx, Ayy, Azz, Axy) (Axz, Ayz, alpha, beta) (live, 1/a_min, - -)
constexpr int kQRec = 4;
constexpr int kSub = 8;  // sub-boxes of a tile in the producer's cull

template <class C>
struct __align__(16) EvalSmem {
    ChunkBlock blk[C::NS][C::CHB];
    SlotMeta meta[C::NS][C::CHB];
    int count[C::NS];
    int abort;  // an earlier launch on this stream timed out: skip the work
    int active; // flags mode: consumer warps with an unsettled primitive
    int pad[2];
    uint64_t full[C::NS];
    uint64_t empty[C::NS];
    float4 q[C::NCW * C::QW][kQRec];
    // the producer's sub-boxes: rows [k TQ/kSub, (k + 1) TQ/kSub) of the tile,
    // (min centre, max alpha) (max centre, max beta)
    float4 sub[kSub][2];
    // spheres, each value duplicated for packed evaluation against two
    // Gaussians at once: (-cx, -cx, -cy, -cy) (-cz, -cz, 1/r^2, 1/r^2) (-2n, -2n, 0, 0)
    float4 qd[C::NCW * C::QW][3];
    // per consumer warp: the stage's slots that pass the warp test, by rank
    // (the quad tests of sweep launches)
    int slots[C::NCW][32];
    // per consumer warp: its box of primitive centres with the largest reach
    // parameters, (lo, alpha) (hi, beta), and on the sweep quad shapes each
    // quad as one sphere record (read by the per-stage tests; kept here rather
    // than in registers)
    float4 wbox[C::NCW][2];
    float4 wquad[C::NCW][4][2];
    // persistent shapes: tile indices from the producer to the consumer
    // warps, two deep (tfull: one arrival by the producer; tempty: one per
    // consumer warp once it has read the index)
    uint64_t tfull[2];
    uint64_t tempty[2];
    int tile_q[2];
    // per consumer warp, its kernel counters (cs_params.out_kernel_stats), kept
    // here rather than in registers: stages, slots tested, slots passing the
    // warp test, polls, wait cycles, first-stage wait, start clock
    unsigned long long wst[C::NCW][7];
};

template <int PRIM> struct PrimTraits;
template <> struct PrimTraits<0> { static constexpr int RECS = 1; };  // sphere: (c, r)
template <> struct PrimTraits<1> { static constexpr int RECS = 3; };  // ellipsoid

// Cull parameters of one prepared primitive: every pair whose centre distance
// exceeds alpha*s + sqrt(alpha^2 s^2 + beta) (s = the Gaussian's largest
// scale) has st2 > S_reach.
//   sphere:    alpha = n, beta = S r^2 (|d|^2 - 2 n s |d| <= S r^2; with the
//              exact variance the reach adds the trace term itself);
//   ellipsoid: in the ellipsoid's own scaling t = sqrt(s^2) = |A^1/2 d|,
//              |A d| <= t / a_min, so sqrt(sigma^2) <= 2 s t / a_min and
//              st2 <= S requires t <= t_max(s) = nu s/a_min + sqrt(nu^2 s^2/a_min^2 + S)
//              with nu = n; then |d| <= a_max t_max(s), i.e.
//              alpha = nu a_max/a_min, beta = S a_max^2.  With the exact
//              variance, tr((A Sigma)^2)/2 <= 1.5 s^4/a_min^4 adds at most
//              sqrt(6) n s^2/a_min^2 to the condition on t, which
//              nu = sqrt(n^2 + sqrt(6) n) covers.
// The consumers' per-chunk ellipsoid test (reaches) works with t_max itself.
template <int PRIM, bool EX>
__device__ __forceinline__ void prim_reach(const float4 *rec, float ns, float S, float &alpha, float &beta) {
    if (PRIM == 0) {
        float r = rec[0].w;
        alpha = ns;
        beta = S * r * r;
    } else {
        float amax = rec[0].w, amin = rec[2].z;
        const float nu = EX ? sqrtf(fmaf(ns, ns, 2.4494898f * ns)) : ns;
        alpha = nu * amax / amin;
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
// microseconds).  Each poll may sleep up to kWaitHintNs for the phase.
// Returns the number of polls the wait took, or -1 when it gave up.
constexpr unsigned kWaitHintNs = 20000;
__device__ __noinline__ long long wait_phase(uint64_t *bar, unsigned parity, long long polls) {
    long long t0 = globaltimer_ns();
    for (long long i = 0; i < polls; ++i) {
        if (mbar_try_wait_hint(bar, parity, kWaitHintNs)) return i + 1;
        if ((i & 255) == 255 && globaltimer_ns() - t0 > 1000000000ll) break;
    }
    return -1;
}


// ------------------------------------------------------------- producer
template <int PRIM, class C, bool EX>
struct Producer {
    EvalSmem<C> *sm;
    const SceneDev *sc;
    long long polls;
    float lx, ly, lz, hx, hy, hz, al, be;  // tile box and reach parameters
    int k = 0;       // stage sequence number
    int nslot = 0;   // chunk slots filled in the open stage
    bool failed = false;
    unsigned *err = nullptr;  // the stream's error word (index checks of CS_DEBUG builds)
    bool early = false;   // flags mode: stop staging once every consumer warp is settled
    bool halted = false;
    int lane;
    unsigned long long n_chunks = 0, n_polls = 0, n_wait_cycles = 0, t_first = 0;
    long long t0 = 0;

    __device__ void open_stage() {
        int s = k % C::NS;
        if (k >= C::NS) {
            bool ok = true;
            if (lane == 0) {
                const long long c0 = clock64();
                const long long w = wait_phase(&sm->empty[s], (unsigned)((k / C::NS - 1) & 1), polls);
                n_wait_cycles += (unsigned long long)(clock64() - c0);
                ok = w >= 0;
                n_polls += ok ? (unsigned long long)w : 0ull;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) failed = true;
        }
        nslot = 0;
    }
    __device__ void close_stage() {
        int s = k % C::NS;
        __syncwarp();  // slot metadata written by other lanes before the release
        if (lane == 0) {
            sm->count[s] = nslot;
            mbar_arrive(&sm->full[s]);
            if (k == 0) t_first = (unsigned long long)(clock64() - t0);
        }
        __syncwarp();
        ++k;
        open_stage();
    }
    // Stage chunks [c, c + len) (contiguous blocks); slot metadata carries
    // each chunk's index and its number of real slots.
    __device__ void emit_run(int c, int len) {
        if (early && !halted) halted = __shfl_sync(0xffffffffu, *(volatile int *)&sm->active == 0, 0);
        if (!CS_IDX_OK(c >= 0 && len >= 0 && c + len <= sc->nchunks, err)) len = 0;  // stage nothing
        while (len > 0 && !failed && !halted) {
            const int st = k % C::NS;
            const int take = min(len, C::CHB - nslot);
            if (lane < take) {
                const int cc = c + lane;
                const int nreal = (int)__ldg(&sc->chead[cc].hi.w);
                sm->meta[st][nslot + lane] = SlotMeta{cc, 0, nreal, 0};
            }
            if (lane == 0) {
                unsigned bytes = (unsigned)take * (unsigned)sizeof(ChunkBlock);
                mbar_expect_tx(&sm->full[st], bytes);
                bulk_g2s(&sm->blk[st][nslot], sc->blocks + c, bytes, &sm->full[st]);
            }
            nslot += take;
            n_chunks += (unsigned long long)take;
            c += take;
            len -= take;
            if (nslot == C::CHB) close_stage();
        }
    }
    // Does the tile box + reach meet a chunk or tree node?
    // The tile box first, then its kSub sub-boxes of consecutive rows: a
    // sparse tile (primitives scattered over the scene) stages only what
    // some group of its rows can reach.
    __device__ bool meets(const NodeBox &b) const {
        const float R = reach<EX && PRIM == 0>(al, be, b.lo.w, sc->pad_abs);
        if (box_gap2(lx, ly, lz, hx, hy, hz, b.lo, b.hi) > R * R) return false;
#pragma unroll 1
        for (int k = 0; k < kSub; ++k) {
            const float4 lo = sm->sub[k][0], hi = sm->sub[k][1];
            const float Rk = reach<EX && PRIM == 0>(lo.w, hi.w, b.lo.w, sc->pad_abs);
            if (box_gap2(lo.x, lo.y, lo.z, hi.x, hi.y, hi.z, b.lo, b.hi) <= Rk * Rk) return true;
        }
        return false;
    }
    // Lane-parallel test of the up to 32 records [base, base + 32) of `recs`.
    __device__ unsigned test32(const NodeBox *recs, int base, int count) const {
        const int i = base + lane;
        bool hit = false;
        if (i < count) hit = meets(recs[i]);
        return __ballot_sync(0xffffffffu, hit);
    }
    // Descend the chunk tree from the top level and stage every chunk whose
    // box + reach meets the tile box, in increasing chunk order (runs of
    // consecutive passing chunks are one bulk copy each).
    __device__ void descend() {
        const int n3 = sc->nnodes[2], n2 = sc->nnodes[1], n1 = sc->nnodes[0], nc = sc->nchunks;
        for (int b3 = 0; b3 < n3 && !failed && !halted; b3 += 32) {
            unsigned m3 = test32(sc->nodes[2], b3, n3);
            while (m3 && !failed && !halted) {
                const int i3 = b3 + __ffs(m3) - 1;
                m3 &= m3 - 1;
                unsigned m2 = test32(sc->nodes[1], 32 * i3, n2);
                while (m2 && !failed && !halted) {
                    const int i2 = 32 * i3 + __ffs(m2) - 1;
                    m2 &= m2 - 1;
                    unsigned m1 = test32(sc->nodes[0], 32 * i2, n1);
                    while (m1 && !failed && !halted) {
                        const int i1 = 32 * i2 + __ffs(m1) - 1;
                        m1 &= m1 - 1;
                        unsigned mc = test32(sc->chead, 32 * i1, nc);
                        while (mc && !failed && !halted) {
                            const int first = __ffs(mc) - 1;
                            const unsigned rest = ~(mc >> first);
                            const int len = rest ? __ffs(rest) - 1 : 32 - first;
                            emit_run(32 * i1 + first, len);
                            mc = (first + len >= 32) ? 0u : (mc & ~((1u << (first + len)) - 1u));
                        }
                    }
                }
            }
        }
    }
    __device__ void finish() {
        if (failed) return;
        if (nslot > 0) close_stage();
        if (failed) return;
        int s = k % C::NS;
        if (lane == 0) {
            sm->count[s] = 0;  // terminator
            mbar_arrive(&sm->full[s]);
        }
        __syncwarp();
    }
    // Persistent shapes: end the tile with a terminator stage and open the
    // next stage of the ring (the consumers release terminators too).
    __device__ void finish_tile() {
        if (failed) return;
        if (nslot > 0) close_stage();
        if (failed) return;
        const int s = k % C::NS;
        if (lane == 0) {
            sm->count[s] = 0;  // terminator
            mbar_arrive(&sm->full[s]);
        }
        __syncwarp();
        ++k;
        open_stage();
    }
    // After a failed wait: close the open stage so its copies can complete,
    // then wait (bounded) for every stage's latest phase.
    __device__ void drain() {
        __syncwarp();
        if (lane == 0) {
            int s = k % C::NS;
            if (nslot > 0) {
                sm->count[s] = nslot;
                mbar_arrive(&sm->full[s]);
                ++k;
            }
            for (int j = max(0, k - C::NS); j < k; ++j)
                wait_phase(&sm->full[j % C::NS], (unsigned)((j / C::NS) & 1), polls);
        }
        __syncwarp();
    }
};

// The tile's box of primitive centres and its largest reach parameters
// (alpha, beta), warp-wide, and its kSub sub-boxes of consecutive rows into
// shared memory (read by the producer's cull only).
template <int PRIM, class C, bool EX>
__device__ __forceinline__ void tile_bounds(const EvalArgs &a, EvalSmem<C> *sm, int tile, int lane, float &lx,
                                            float &ly, float &lz, float &hx, float &hy, float &hz, float &al,
                                            float &be) {
    constexpr int RECS = PrimTraits<PRIM>::RECS;
    constexpr int TQ = C::NCW * C::QW;
    lx = INFINITY; ly = INFINITY; lz = INFINITY; hx = -INFINITY; hy = -INFINITY; hz = -INFINITY;
    al = 0.f; be = 0.f;
    const int q0 = tile * TQ;
    constexpr int RS = TQ / kSub;  // rows per sub-box (4, 8 or 16: within one pass of 32 lanes)
    static_assert(TQ % kSub == 0 && RS <= 32 && 32 % RS == 0, "sub-boxes split the tile's rows evenly");
#pragma unroll
    for (int t0 = 0; t0 < TQ; t0 += 32) {
        const int t = t0 + lane, q = q0 + t;
        float cx = INFINITY, cy = INFINITY, cz = INFINITY, dx = -INFINITY, dy = -INFINITY, dz = -INFINITY;
        float alpha = 0.f, beta = 0.f;
        if (t < TQ && q < a.Q) {
            const float4 *rec = row_rec<RECS>(a, q);
            const float4 r0 = rec[0];
            if (rec_valid(r0)) {
                prim_reach<PRIM, EX>(rec, row_ns(a, q), a.k.S_reach, alpha, beta);
                cx = dx = r0.x; cy = dy = r0.y; cz = dz = r0.z;
            }
        }
        lx = fminf(lx, cx); ly = fminf(ly, cy); lz = fminf(lz, cz);
        hx = fmaxf(hx, dx); hy = fmaxf(hy, dy); hz = fmaxf(hz, dz);
        al = fmaxf(al, alpha);
        be = fmaxf(be, beta);
        // sub-box of the RS consecutive rows of this lane's group
#pragma unroll
        for (int o = RS / 2; o > 0; o >>= 1) {
            cx = fminf(cx, __shfl_xor_sync(0xffffffffu, cx, o));
            cy = fminf(cy, __shfl_xor_sync(0xffffffffu, cy, o));
            cz = fminf(cz, __shfl_xor_sync(0xffffffffu, cz, o));
            dx = fmaxf(dx, __shfl_xor_sync(0xffffffffu, dx, o));
            dy = fmaxf(dy, __shfl_xor_sync(0xffffffffu, dy, o));
            dz = fmaxf(dz, __shfl_xor_sync(0xffffffffu, dz, o));
            alpha = fmaxf(alpha, __shfl_xor_sync(0xffffffffu, alpha, o));
            beta = fmaxf(beta, __shfl_xor_sync(0xffffffffu, beta, o));
        }
        if (t < TQ && lane % RS == 0) {
            sm->sub[t / RS][0] = make_float4(cx, cy, cz, alpha);
            sm->sub[t / RS][1] = make_float4(dx, dy, dz, beta);
        }
    }
    __syncwarp();
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
}

template <int PRIM, class C, bool EX>
__device__ void producer_warp(const EvalArgs &a, EvalSmem<C> *sm, int tile, bool early) {
    const int lane = threadIdx.x & 31;
    const long long t_start = clock64();
    const SceneDev &sc = a.sc;
    float lx, ly, lz, hx, hy, hz, al, be;
    tile_bounds<PRIM, C, EX>(a, sm, tile, lane, lx, ly, lz, hx, hy, hz, al, be);
    Producer<PRIM, C, EX> pr{sm, &sc, a.wait_polls, lx, ly, lz, hx, hy, hz, al, be};
    pr.early = early;
    pr.err = a.err;
    pr.lane = lane;
    pr.t0 = t_start;
    const bool any = lx <= hx;  // at least one valid primitive
    if (any && sc.nchunks > 0) pr.descend();
    pr.finish();
    if (pr.failed) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        pr.drain();
    }
    if (a.kstats && lane == 0) {
        atomicAdd(a.kstats + 4, pr.n_chunks);
        atomicAdd(a.kstats + 5, (unsigned long long)pr.k);
        atomicAdd(a.kstats + 7, pr.n_polls);
        atomicAdd(a.kstats + 10, (unsigned long long)(clock64() - t_start));
        atomicAdd(a.kstats + 11, pr.n_wait_cycles);
        atomicAdd(a.kstats + 13, pr.t_first);
        atomicAdd(a.kstats + 15, 1ull);
    }
}

// Persistent shapes: the producer takes tile after tile from the launch's
// counter, hands each index to the consumer warps through the two-deep tile
// queue (tile_q), and culls and stages it; the consumers' terminator releases
// close each tile.  A final index >= ntiles (or -1 after a failed wait) ends
// the consumers.
template <int PRIM, class C, bool EX>
__device__ void producer_persistent(const EvalArgs &a, EvalSmem<C> *sm) {
    const int lane = threadIdx.x & 31;
    const long long t_start = clock64();
    const SceneDev &sc = a.sc;
    Producer<PRIM, C, EX> pr{sm, &sc, a.wait_polls, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    pr.err = a.err;
    pr.lane = lane;
    pr.t0 = t_start;
    unsigned long long tiles = 0;
    for (int i = 0;; ++i) {
        int tile = 0;
        if (lane == 0) tile = atomicAdd(a.tile_ctr, 1);
        tile = __shfl_sync(0xffffffffu, tile, 0);
        const int slot = i & 1;
        bool ok = true;
        if (i >= 2 && lane == 0)  // the consumers have read index i - 2 from this slot
            ok = wait_phase(&sm->tempty[slot], (unsigned)(((i >> 1) - 1) & 1), a.wait_polls) >= 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) pr.failed = true;
        if (lane == 0) {
            sm->tile_q[slot] = pr.failed ? -1 : tile;
            mbar_arrive(&sm->tfull[slot]);  // release: the index is visible to the waiting consumers
        }
        __syncwarp();
        if (pr.failed || tile >= a.ntiles) break;
        tile_bounds<PRIM, C, EX>(a, sm, tile, lane, pr.lx, pr.ly, pr.lz, pr.hx, pr.hy, pr.hz, pr.al, pr.be);
        if (pr.lx <= pr.hx && sc.nchunks > 0) pr.descend();
        pr.finish_tile();
        ++tiles;
        if (pr.failed) break;
    }
    if (pr.failed) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        pr.drain();
    }
    if (a.kstats && lane == 0) {
        atomicAdd(a.kstats + 4, pr.n_chunks);
        atomicAdd(a.kstats + 5, (unsigned long long)pr.k);
        atomicAdd(a.kstats + 7, pr.n_polls);
        atomicAdd(a.kstats + 10, (unsigned long long)(clock64() - t_start));
        atomicAdd(a.kstats + 11, pr.n_wait_cycles);
        atomicAdd(a.kstats + 13, pr.t_first);
        atomicAdd(a.kstats + 15, tiles);
    }
}

// ------------------------------------------------------------- consumers
// MODE: 0 = cost (mean/sum), 1 = min, 2 = softmin, 3 = collision flags only.
// A consumer warp owns QW primitives.  Lane l takes Gaussian l of every
// staged chunk (global sorted index 32c + l), so each lane's partial
// reductions run over a fixed subsequence of the scene in increasing order,
// whatever the tile: results do not depend on which rows share the launch.
template <int PRIM, int QW, int MODE, bool GRAD>
struct Acc {
    // cost partial over the current chunk group (ellipsoids; spheres sum directly)
    float sumb[(MODE == 0 && !GRAD && PRIM == 1) ? QW : 1];
    float sum[(MODE == 0) ? QW : 1];  // (adjoint: only with kShFwd)
    float mn[(MODE == 1) ? QW : 1];
    float sm_m[(MODE == 2) ? QW : 1];
    float sm_acc[(MODE == 2) ? QW : 1];
    float gx[GRAD ? QW : 1], gy[GRAD ? QW : 1], gz[GRAD ? QW : 1];
    int cnt[MODE == 3 ? 1 : QW];
    int cin[(GRAD && PRIM == 1) ? 1 : QW];
    // sphere cost launches with k_thr = 0: bit j is set once a pair of row j
    // has st2 < T_in (the row collides iff a lane set it), in place of the
    // in-collision count
    unsigned fin;
};

// Lane-local Gaussian of the current chunk slot (f: tr(Sigma^2)/2, set for
// spheres with the exact variance only).
struct LaneG {
    float x, y, z, sxx, syy, szz, sxy2, sxz2, syz2, f;
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// tr((A Sigma)^2) / 2 for an ellipsoid record (A symmetric) and a Gaussian:
// with P = A Sigma, tr(P P) = sum_i P_ii^2 + 2 sum_{i<j} P_ij P_ji.
__device__ __forceinline__ float half_tr_asas(const float4 *qd, const LaneG &g) {
    const float axx = qd[1].x, ayy = qd[1].y, azz = qd[1].z, axy = qd[1].w, axz = qd[2].x, ayz = qd[2].y;
    const float hxy = 0.5f * g.sxy2, hxz = 0.5f * g.sxz2, hyz = 0.5f * g.syz2;
    const float p00 = fmaf(axz, hxz, fmaf(axy, hxy, axx * g.sxx));
    const float p01 = fmaf(axz, hyz, fmaf(axy, g.syy, axx * hxy));
    const float p02 = fmaf(axz, g.szz, fmaf(axy, hyz, axx * hxz));
    const float p10 = fmaf(ayz, hxz, fmaf(ayy, hxy, axy * g.sxx));
    const float p11 = fmaf(ayz, hyz, fmaf(ayy, g.syy, axy * hxy));
    const float p12 = fmaf(ayz, g.szz, fmaf(ayy, hyz, axy * hxz));
    const float p20 = fmaf(azz, hxz, fmaf(ayz, hxy, axz * g.sxx));
    const float p21 = fmaf(azz, hyz, fmaf(ayz, g.syy, axz * hxy));
    const float p22 = fmaf(azz, g.szz, fmaf(ayz, hyz, axz * hxz));
    const float diag = fmaf(p22, p22, fmaf(p11, p11, p00 * p00));
    const float off = fmaf(p12, p21, fmaf(p02, p20, p01 * p10));
    return fmaf(0.5f, diag, off);
}

// tr(Sigma^2)/2 of a Gaussian from its doubled off-diagonals (the exact
// variance's trace term for a sphere, before the 1/r^2 scaling).
__device__ __forceinline__ float half_tr_ss(const LaneG &g) {
    return fmaf(0.25f, fmaf(g.syz2, g.syz2, fmaf(g.sxz2, g.sxz2, g.sxy2 * g.sxy2)),
                0.5f * fmaf(g.szz, g.szz, fmaf(g.syy, g.syy, g.sxx * g.sxx)));
}

// One (primitive, Gaussian) pair.  EX: sigma^2 is the exact variance of the
// quadratic form, 4 w^T Sigma w + 2 tr((A Sigma)^2), i.e. u + tr((A Sigma)^2)/2
// under the root (for a sphere A = I / r^2 and the trace term is the lane's
// g.f = tr(Sigma^2)/2, scaled by 1/r^2 with the rest).
template <int PRIM, int QW, int MODE, bool GRAD, bool EX = false, bool FWD = false>
__device__ __forceinline__ void pair_update(Acc<PRIM, QW, MODE, GRAD> &A, int j, const LaneG &g,
                                            const float4 *qd, const QueryConsts &k) {
    const float dx = g.x - qd[0].x, dy = g.y - qd[0].y, dz = g.z - qd[0].z;
    float s2, u, vx = 0.f, vy = 0.f, vz = 0.f;   // s2: Eq. 5 numerator (sphere) or Eq. 5
    float ns2, ir2;
    float wx = dx, wy = dy, wz = dz;             // w = A d (sphere: d, scaled by 1/r^2 later)
    if (PRIM == 0) {
        ns2 = qd[1].x;
        ir2 = qd[0].w;
        s2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    } else {
        ns2 = qd[0].w;
        ir2 = 1.f;
        const float axx = qd[1].x, ayy = qd[1].y, azz = qd[1].z, axy = qd[1].w, axz = qd[2].x, ayz = qd[2].y;
        wx = fmaf(axz, dz, fmaf(axy, dy, axx * dx));
        wy = fmaf(ayz, dz, fmaf(ayy, dy, axy * dx));
        wz = fmaf(azz, dz, fmaf(ayz, dy, axz * dx));
        s2 = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
    }
    float F = 0.f;  // EX: the trace term, added first (the packed path does the same)
    if constexpr (EX) F = (PRIM == 0) ? g.f : half_tr_asas(qd, g);
    if (!GRAD) {
        // w^T Sigma w with the doubled off-diagonals: 9 FP32 ops
        const float t1 = fmaf(g.sxz2, wz, fmaf(g.sxy2, wy, g.sxx * wx));
        const float t2 = fmaf(g.syz2, wz, g.syy * wy);
        u = fmaf(wx, t1, fmaf(wy, t2, EX ? fmaf(wz, g.szz * wz, F) : wz * (g.szz * wz)));
    } else {
        const float hxy = 0.5f * g.sxy2, hxz = 0.5f * g.sxz2, hyz = 0.5f * g.syz2;
        vx = fmaf(hxz, wz, fmaf(hxy, wy, g.sxx * wx));  // Sigma w
        vy = fmaf(hyz, wz, fmaf(g.syy, wy, hxy * wx));
        vz = fmaf(g.szz, wz, fmaf(hyz, wy, hxz * wx));
        u = fmaf(wx, vx, fmaf(wy, vy, EX ? fmaf(wz, vz, F) : wz * vz));
    }
    u = fmaxf(u, 0.f);
    float sq, rsq = 0.f;
    if (!GRAD) {
        sq = sqrt_approx(u);
    } else {
        rsq = u > 0.f ? rsqrtf(u) : 0.f;
        sq = u * rsq;
    }
    // Eq. 8: st2 = max(0, s^2 - n sqrt(sigma^2)); for a sphere s^2 and
    // sqrt(sigma^2) = 2 sqrt(d^T Sigma d)/r^2 share the factor 1/r^2.
    const float raw = fmaf(-ns2, sq, s2);
    // Eq. 8 clamp.  For an ellipsoid with a large A, d^T A d of a padding
    // point (at 1e18) overflows: a first product of either sign becomes +-inf
    // (or NaN), which the clamp would turn into 0, a colliding neighbour.
    // d^T A d >= 0, so a non-finite value can only be an overflow: it counts
    // as +inf (beyond every threshold), and padding still adds nothing.
    const float st2 = (PRIM == 0 ? fmaxf(raw, 0.f) : (fabsf(raw) <= FLT_MAX ? fmaxf(raw, 0.f) : INFINITY)) * ir2;
    if constexpr (MODE == 3) {  // flags only: the in-collision count (Section II-E)
        A.cin[j] += (st2 < k.T_in) ? 1 : 0;
    } else {
        // Eq. 11 without d_max (applied once per primitive): 2^min(-G (st2 - s_min), 0)
        const float dc = ex2_approx(fminf(fmaf(st2, -k.G, k.Gsmin), 0.f));
        const bool nb = st2 <= k.S_cut;
        A.cnt[j] += nb ? 1 : 0;
        if (!GRAD) {
            A.cin[j] += (st2 < k.T_in) ? 1 : 0;
            if (MODE == 0) {
                if (PRIM == 1) A.sumb[j] += nb ? dc : 0.f;
                else A.sum[j] += nb ? dc : 0.f;
            }
            if (MODE == 1) A.mn[j] = fminf(A.mn[j], st2);
            if (MODE == 2) {
                const float nm = nb ? fminf(A.sm_m[j], st2) : A.sm_m[j];
                const float f = ex2_approx((nm - A.sm_m[j]) * k.K);
                const float e = nb ? ex2_approx((nm - st2) * k.K) : 0.f;
                A.sm_acc[j] = fmaf(A.sm_acc[j], f, e);
                A.sm_m[j] = nm;
            }
        } else {
            // d st2 / d c = (-2 w + 2 n A Sigma w / sqrt(w^T Sigma w)) * ir2 where raw > 0
            float px = vx, py = vy, pz = vz;
            if (PRIM == 1) {
                const float axx = qd[1].x, ayy = qd[1].y, azz = qd[1].z, axy = qd[1].w, axz = qd[2].x, ayz = qd[2].y;
                px = fmaf(axz, vz, fmaf(axy, vy, axx * vx));
                py = fmaf(ayz, vz, fmaf(ayy, vy, axy * vx));
                pz = fmaf(azz, vz, fmaf(ayz, vy, axz * vx));
            }
            const float rs = ns2 * rsq;
            const float live = raw > 0.f ? ir2 : 0.f;
            const float ex = fmaf(rs, px, -2.f * wx) * live;
            const float ey = fmaf(rs, py, -2.f * wy) * live;
            const float ez = fmaf(rs, pz, -2.f * wz) * live;
            if (MODE == 0) {
                if constexpr (FWD && PRIM == 0) {  // the forward reductions of the same pair
                    A.cin[j] += (st2 < k.T_in) ? 1 : 0;
                    A.sum[j] += nb ? dc : 0.f;
                }
                // Eq. 11 is flat (zero gradient) below s_min
                const float w = (nb && st2 > k.s_min) ? dc : 0.f;
                A.gx[j] = fmaf(w, ex, A.gx[j]);
                A.gy[j] = fmaf(w, ey, A.gy[j]);
                A.gz[j] = fmaf(w, ez, A.gz[j]);
            } else if (MODE == 1) {
                const bool take = nb && st2 < A.mn[j];
                A.mn[j] = take ? st2 : A.mn[j];
                A.gx[j] = take ? ex : A.gx[j];
                A.gy[j] = take ? ey : A.gy[j];
                A.gz[j] = take ? ez : A.gz[j];
            } else {
                const float nm = nb ? fminf(A.sm_m[j], st2) : A.sm_m[j];
                const float f = ex2_approx((nm - A.sm_m[j]) * k.K);
                const float e = nb ? ex2_approx((nm - st2) * k.K) : 0.f;
                A.sm_acc[j] = fmaf(A.sm_acc[j], f, e);
                A.gx[j] = fmaf(A.gx[j], f, e * ex);
                A.gy[j] = fmaf(A.gy[j], f, e * ey);
                A.gz[j] = fmaf(A.gz[j], f, e * ez);
                A.sm_m[j] = nm;
            }
        }
    }
}

// Does the primitive (shared-memory record) reach the chunk (bounding box,
// largest scale)?  Dead slots never do.  The same answer on every lane.
template <int PRIM, bool EX>
__device__ __forceinline__ bool reaches(const float4 *qd, const float4 &blo, const float4 &bhi,
                                        float pad_abs, float S) {
    const float4 q0 = qd[0];
    if (PRIM == 0) {
        const float4 q1 = qd[1];
        const float R = reach<EX>(q1.y, q1.z, blo.w, pad_abs);
        return q1.w != 0.f && box_gap2(q0.x, q0.y, q0.z, q0.x, q0.y, q0.z, blo, bhi) <= R * R;
    } else {
        // In the ellipsoid's scaling t = |A^1/2 (x - c)|, which changes by at
        // most |x - y| / a_min between two points: every point of the chunk's
        // box lies within its half-diagonal rho of the box centre b, so a pair
        // of the chunk can be within reach only if
        //   t(b) <= t_max(sigma) + (rho + pad) / a_min,
        // t_max the largest t with t^2 - 2 n sqrt(tau^2 t^2 [+ 1.5 tau^4]) <= S,
        // tau = sigma / a_min (the bracket with the exact variance): the
        // sphere reach in the ellipsoid's own scaling (reach with alpha = n,
        // beta = S), checked with a relative margin for the FP32 rounding of
        // t(b)^2.
        const float4 q1 = qd[1], q2 = qd[2], q3 = qd[3];
        const float inv_amin = q3.y;
        const float dx = fmaf(0.5f, blo.x + bhi.x, -q0.x), dy = fmaf(0.5f, blo.y + bhi.y, -q0.y),
                    dz = fmaf(0.5f, blo.z + bhi.z, -q0.z);
        const float ex = bhi.x - blo.x, ey = bhi.y - blo.y, ez = bhi.z - blo.z;
        const float rho = 0.5f * sqrtf(fmaf(ez, ez, fmaf(ey, ey, ex * ex)));
        const float wx = fmaf(q2.x, dz, fmaf(q1.w, dy, q1.x * dx));
        const float wy = fmaf(q2.y, dz, fmaf(q1.y, dy, q1.w * dx));
        const float wz = fmaf(q1.z, dz, fmaf(q2.y, dy, q2.x * dx));
        const float t2 = fmaf(dz, wz, fmaf(dy, wy, dx * wx));
        const float tmax = reach<EX>(0.5f * q0.w, S, blo.w * inv_amin, 0.f);
        const float T = fmaf(rho + pad_abs, inv_amin, tmax) * (1.f + 1e-3f);
        return q3.x != 0.f && t2 <= T * T;
    }
}

// Lane-local Gaussian duplicated into both halves of packed registers.
struct LaneG2 {
    f32x2 x, y, z, sxx, syy, szz, sxy2, sxz2, syz2, f;
};

// One sphere (cost reductions, forward) against the lane's two Gaussians
// (one from each chunk of a chunk pair), with the geometry of Eq. 5, 7, 8 and
// the Eq. 11 exponent in packed FP32x2: the operations of pair_update in
// its order (less the clamp of Eq. 8, which tail_g2 replaces exactly), hence
// the same bits; half 0 is accumulated before half 1, so each lane still
// adds its Gaussians in increasing order.
// The geometry part: |d|^2 and sqrt(d^T Sigma d [+ trace term]) for the
// sphere of `qd` and the lane's two Gaussians (it depends on the sphere's
// centre only, not on its n_sigma).
template <bool EX>
__device__ __forceinline__ void geom_g2(const LaneG2 &g, const float4 *qd, f32x2 &r2, f32x2 &sq) {
    const ulonglong2 pa = *reinterpret_cast<const ulonglong2 *>(&qd[0]);  // -cx, -cy
    const ulonglong2 pb = *reinterpret_cast<const ulonglong2 *>(&qd[1]);  // -cz, 1/r^2
    const f32x2 dx = add2(g.x, pa.x), dy = add2(g.y, pa.y), dz = add2(g.z, pb.x);
    r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const f32x2 t1 = fma2(g.sxz2, dz, fma2(g.sxy2, dy, mul2(g.sxx, dx)));
    const f32x2 t2 = fma2(g.syz2, dz, mul2(g.syy, dy));
    const f32x2 zz = mul2(g.szz, dz);
    const f32x2 u = fma2(dx, t1, fma2(dy, t2, EX ? fma2(dz, zz, g.f) : mul2(dz, zz)));
    float u0, u1;
    upk2(u, u0, u1);
    sq = pk2(sqrt_approx(fmaxf(u0, 0.f)), sqrt_approx(fmaxf(u1, 0.f)));
}

// The rest for row j with its own n_sigma (qd[2]) and scale (qd[1]).
// st2 is not clamped at 0 here; the outputs still equal those of the clamped
// value bit for bit.  Where st2 >= 0 nothing changes.  Where st2 < 0 (the
// clamped value is 0):
//   - e = -G st2 + G s_min >= G s_min, so min(e, min(G s_min, 0)) is
//     min(G s_min, 0), the capped exponent of st2 = 0 (for st2 >= 0,
//     e <= G s_min and the cap leaves min(e, 0));
//   - st2 <= S_cut_u and st2 < T_in_u hold exactly when 0 <= S_cut and
//     0 < T_in, as for the clamped value.
template <int QW, bool K0>
__device__ __forceinline__ void tail_g2v(Acc<0, QW, 0, false> &A, int j, f32x2 r2, f32x2 sq, f32x2 ir2,
                                         f32x2 nns2, const QueryConsts &k, f32x2 nG2, f32x2 Gs2) {
    const f32x2 st = mul2(fma2(nns2, sq, r2), ir2);
    float e0, e1, s0, s1;
    upk2(fma2(st, nG2, Gs2), e0, e1);
    upk2(st, s0, s1);
    const float dc0 = ex2_approx(fminf(e0, k.E_cap)), dc1 = ex2_approx(fminf(e1, k.E_cap));
    const bool nb0 = s0 <= k.S_cut_u, nb1 = s1 <= k.S_cut_u;
    A.cnt[j] += (nb0 ? 1 : 0) + (nb1 ? 1 : 0);
    if constexpr (K0) {
        A.fin |= (s0 < k.T_in_u || s1 < k.T_in_u) ? (1u << j) : 0u;
    } else {
        A.cin[j] += ((s0 < k.T_in_u) ? 1 : 0) + ((s1 < k.T_in_u) ? 1 : 0);
    }
    A.sum[j] += nb0 ? dc0 : 0.f;
    A.sum[j] += nb1 ? dc1 : 0.f;
}

// The same for row j's record in shared memory: scale (qd[1]) and n_sigma (qd[2]).
template <int QW, bool K0>
__device__ __forceinline__ void tail_g2(Acc<0, QW, 0, false> &A, int j, f32x2 r2, f32x2 sq, const float4 *qd,
                                        const QueryConsts &k, f32x2 nG2, f32x2 Gs2) {
    const ulonglong2 pb = *reinterpret_cast<const ulonglong2 *>(&qd[1]);  // -cz, 1/r^2
    const f32x2 nns2 = *reinterpret_cast<const f32x2 *>(&qd[2]);          // -2n
    tail_g2v<QW, K0>(A, j, r2, sq, pb.y, nns2, k, nG2, Gs2);
}

template <int QW, bool EX, bool K0>
__device__ __forceinline__ void pair_update_g2(Acc<0, QW, 0, false> &A, int j, const LaneG2 &g,
                                               const float4 *qd, const QueryConsts &k, f32x2 nG2, f32x2 Gs2) {
    f32x2 r2, sq;
    geom_g2<EX>(g, qd, r2, sq);
    tail_g2<QW, K0>(A, j, r2, sq, qd, k, nG2, Gs2);
}

// The adjoint (mean or sum cost, forward reductions too with FWD) of one
// sphere against the lane's two Gaussians in packed FP32x2: the operations
// of pair_update's adjoint body in its order (two scalar IEEE operations per
// packed one, so the same bits), half 0 accumulated before half 1.
template <int QW, bool FWD>
__device__ __forceinline__ void pair_update_g2_grad(Acc<0, QW, 0, true> &A, int j, const LaneG2 &g,
                                                    const float4 *qd, const QueryConsts &k) {
    const ulonglong2 pa = *reinterpret_cast<const ulonglong2 *>(&qd[0]);  // -cx, -cy
    const ulonglong2 pb = *reinterpret_cast<const ulonglong2 *>(&qd[1]);  // -cz, 1/r^2
    const f32x2 nns2 = *reinterpret_cast<const f32x2 *>(&qd[2]);          // -2n
    const f32x2 dx = add2(g.x, pa.x), dy = add2(g.y, pa.y), dz = add2(g.z, pb.x);
    const f32x2 s2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
    const f32x2 half = pk2(0.5f, 0.5f);
    const f32x2 hxy = mul2(half, g.sxy2), hxz = mul2(half, g.sxz2), hyz = mul2(half, g.syz2);
    const f32x2 vx = fma2(hxz, dz, fma2(hxy, dy, mul2(g.sxx, dx)));  // Sigma d
    const f32x2 vy = fma2(hyz, dz, fma2(g.syy, dy, mul2(hxy, dx)));
    const f32x2 vz = fma2(g.szz, dz, fma2(hyz, dy, mul2(hxz, dx)));
    float u0, u1;
    upk2(fma2(dx, vx, fma2(dy, vy, mul2(dz, vz))), u0, u1);
    u0 = fmaxf(u0, 0.f);
    u1 = fmaxf(u1, 0.f);
    const f32x2 rsq = pk2(u0 > 0.f ? rsqrtf(u0) : 0.f, u1 > 0.f ? rsqrtf(u1) : 0.f);
    const f32x2 sq = mul2(pk2(u0, u1), rsq);
    float r0, r1;
    upk2(fma2(nns2, sq, s2), r0, r1);  // Eq. 8 before the clamp
    const f32x2 st = mul2(pk2(fmaxf(r0, 0.f), fmaxf(r1, 0.f)), pb.y);
    float e0, e1, s0, s1;
    upk2(st, s0, s1);
    // No lane holds a neighbour of this row (st2 <= S_cut) among its two
    // Gaussians: every term below adds exactly nothing (weight 0 times a
    // finite gradient term, no count, no in-collision pair since T_in <=
    // S_cut), so the warp skips them; the outputs keep their bits.
    if (!__any_sync(0xffffffffu, s0 <= k.S_cut || s1 <= k.S_cut)) return;
    upk2(fma2(st, pk2(-k.G, -k.G), pk2(k.Gsmin, k.Gsmin)), e0, e1);
    const float dc0 = ex2_approx(fminf(e0, 0.f)), dc1 = ex2_approx(fminf(e1, 0.f));
    const bool nb0 = s0 <= k.S_cut, nb1 = s1 <= k.S_cut;
    A.cnt[j] += (nb0 ? 1 : 0) + (nb1 ? 1 : 0);
    if constexpr (FWD) {
        A.cin[j] += ((s0 < k.T_in) ? 1 : 0) + ((s1 < k.T_in) ? 1 : 0);
        A.sum[j] += nb0 ? dc0 : 0.f;
        A.sum[j] += nb1 ? dc1 : 0.f;
    }
    // d st2 / d c = (-2 d + 2 n Sigma d / sqrt(d^T Sigma d)) / r^2 where the clamp is open
    float ir, ir_dup;
    upk2(pb.y, ir, ir_dup);
    const f32x2 rs = mul2(mul2(nns2, pk2(-1.f, -1.f)), rsq);
    const f32x2 live = pk2(r0 > 0.f ? ir : 0.f, r1 > 0.f ? ir : 0.f);
    const f32x2 m2 = pk2(-2.f, -2.f);
    float ex0, ex1, ey0, ey1, ez0, ez1;
    upk2(mul2(fma2(rs, vx, mul2(m2, dx)), live), ex0, ex1);
    upk2(mul2(fma2(rs, vy, mul2(m2, dy)), live), ey0, ey1);
    upk2(mul2(fma2(rs, vz, mul2(m2, dz)), live), ez0, ez1);
    // Eq. 11 is flat (zero gradient) below s_min
    const float w0 = (nb0 && s0 > k.s_min) ? dc0 : 0.f, w1 = (nb1 && s1 > k.s_min) ? dc1 : 0.f;
    A.gx[j] = fmaf(w0, ex0, A.gx[j]);
    A.gy[j] = fmaf(w0, ey0, A.gy[j]);
    A.gz[j] = fmaf(w0, ez0, A.gz[j]);
    A.gx[j] = fmaf(w1, ex1, A.gx[j]);
    A.gy[j] = fmaf(w1, ey1, A.gy[j]);
    A.gz[j] = fmaf(w1, ez1, A.gz[j]);
}

// Lane l of a staged chunk: its slot l (padding slots already hold a point
// that meets no primitive); an absent chunk (mt.hi == 0) gives that point on
// every lane.
__device__ __forceinline__ void lane_gaussian(const ChunkBlock &B, const SlotMeta mt, int lane, LaneG &g) {
    if (mt.hi > 0) {
        g.x = B.x[lane]; g.y = B.y[lane]; g.z = B.z[lane];
        g.sxx = B.sxx[lane]; g.syy = B.syy[lane]; g.szz = B.szz[lane];
        g.sxy2 = B.sxy2[lane]; g.sxz2 = B.sxz2[lane]; g.syz2 = B.syz2[lane];
    } else {
        g.x = 1e18f; g.y = 1e18f; g.z = 1e18f;
        g.sxx = 0.f; g.syy = 0.f; g.szz = 0.f;
        g.sxy2 = 0.f; g.sxz2 = 0.f; g.syz2 = 0.f;
    }
}

// Two staged chunks (B1 may be absent, mt1.hi == 0) against the spheres of
// `qmask` (the primitives reaching either chunk): lane l holds Gaussian l of
// each chunk in the two halves of packed registers; spheres are evaluated in
// groups of GROUP (a member reaching neither chunk adds exactly nothing).
template <int QW, int GROUP, bool EX, int SH, bool QUAD>
__device__ __forceinline__ void eval_chunk_pair(Acc<0, QW, 0, false> &A, const ChunkBlock &B0, const SlotMeta mt0,
                                                const ChunkBlock &B1, const SlotMeta mt1, unsigned qmask,
                                                float4 (*wqd)[3], const QueryConsts &k, int lane,
                                                unsigned &cand, unsigned &c_hits, unsigned same, unsigned link) {
    constexpr bool K0 = (SH & kShK0) != 0;
    if (qmask == 0u) return;
    LaneG g0, g1;
    lane_gaussian(B0, mt0, lane, g0);
    lane_gaussian(B1, mt1, lane, g1);
    LaneG2 g2;
    g2.x = pk2(g0.x, g1.x); g2.y = pk2(g0.y, g1.y); g2.z = pk2(g0.z, g1.z);
    g2.sxx = pk2(g0.sxx, g1.sxx); g2.syy = pk2(g0.syy, g1.syy); g2.szz = pk2(g0.szz, g1.szz);
    g2.sxy2 = pk2(g0.sxy2, g1.sxy2); g2.sxz2 = pk2(g0.sxz2, g1.sxz2); g2.syz2 = pk2(g0.syz2, g1.syz2);
    if constexpr (EX) g2.f = pk2(half_tr_ss(g0), half_tr_ss(g1));
    const f32x2 nG2 = pk2(-k.G, -k.G), Gs2 = pk2(k.Gsmin, k.Gsmin);
    // bit j0 of gm: group j0 .. j0 + GROUP - 1 has a member reaching a chunk
    unsigned gm = qmask;
#pragma unroll
    for (int sh = 1; sh < GROUP; sh <<= 1) gm |= gm >> sh;
    constexpr unsigned LEAD = GROUP == 1 ? 0xFFFFFFFFu : GROUP == 2 ? 0x55555555u : GROUP == 4 ? 0x11111111u
                                                                               : 0x01010101u;
    gm &= LEAD;
    const unsigned ng = (unsigned)__popc(gm) * (unsigned)GROUP;
    c_hits += ng;
    cand += ng * (unsigned)((mt0.hi - mt0.lo) + (mt1.hi - mt1.lo));
    // geometry of the last group evaluated through the shared branch
    f32x2 r2, sq;
    bool have = false;
#pragma unroll
    for (int j0 = 0; j0 < QW; j0 += GROUP) {
        if ((gm >> j0) & 1u) {
            if ((SH & kShQuad) ||
                ((SH & kShGeom) && GROUP == 4 && ((same >> j0) & (same >> (j0 + 2)) & (link >> (j0 + 2)) & 1u))) {
                // rows j0 .. j0 + 3 are one sphere: the geometry once, four tails
                geom_g2<EX>(g2, wqd[j0], r2, sq);
                // The quad's highest n_sigma copy first.  st2 does not increase
                // with n_sigma, in FP32 too (fma is monotone in each operand and
                // the scale 1/r^2 is positive), so when no lane holds a neighbour
                // of that copy (st2 <= S_cut), no copy has a neighbour or an
                // in-collision pair among these Gaussians (st2 < T_in implies
                // st2 <= S_cut), and the four tails would add exactly nothing.
                // The four rows are one sphere: its scale 1/r^2 (row j0's) serves
                // every tail; each row keeps its own n_sigma.
                const f32x2 ir2 = reinterpret_cast<const ulonglong2 *>(&wqd[j0][1])->y;  // 1/r^2
                {
                    const f32x2 nmax = *reinterpret_cast<const f32x2 *>(&wqd[j0][2].z);  // -2 n_max
                    float t0, t1;
                    upk2(mul2(fma2(nmax, sq, r2), ir2), t0, t1);
                    if (!__any_sync(0xffffffffu, t0 <= k.S_cut_u || t1 <= k.S_cut_u)) continue;
                }
#pragma unroll
                for (int j = j0; j < j0 + 4; ++j)
                    tail_g2v<QW, K0>(A, j, r2, sq, ir2, *reinterpret_cast<const f32x2 *>(&wqd[j][2]), k, nG2, Gs2);
            } else if constexpr ((SH & kShQuad) != 0) {
                // not reached: every group is a quad
            } else if ((SH & kShGeom) && GROUP == 2 && ((same >> j0) & 1u)) {
                // rows j0 and j0 + 1 are the same sphere (n_sigma copies of a
                // sweep): the geometry once, then each row's own n_sigma; the
                // same operations per row as apart, hence the same bits.
                // With QUAD, the geometry of group j0 - 2 serves this group
                // too when row j0 - 1 is the same sphere as row j0.
                if (!(QUAD && have && ((link >> j0) & 1u))) geom_g2<EX>(g2, wqd[j0], r2, sq);
                tail_g2<QW, K0>(A, j0, r2, sq, wqd[j0], k, nG2, Gs2);
                tail_g2<QW, K0>(A, j0 + 1, r2, sq, wqd[j0 + 1], k, nG2, Gs2);
                have = true;
            } else {
#pragma unroll
                for (int j = j0; j < j0 + GROUP; ++j) pair_update_g2<QW, EX, K0>(A, j, g2, wqd[j], k, nG2, Gs2);
                have = false;
            }
        } else {
            have = false;
        }
    }
}

// Sweep launches with whole quads (kShQuad): one chunk pair against the
// warp's quads of `qm` (bit qq: quad qq, rows 4 qq .. 4 qq + 3, reaches
// either chunk).  The operations, and their order per lane and row, are those
// of eval_chunk_pair's quad branch, hence the same bits.  n1 == 0: no second
// chunk (its half holds the padding point, which meets no primitive).
template <int QW, bool EX, int SH>
__device__ __forceinline__ void eval_pair_quads(Acc<0, QW, 0, false> &A, const ChunkBlock &B0, int n0,
                                                const ChunkBlock &B1, int n1, unsigned qm, float4 (*wqd)[3],
                                                const QueryConsts &k, int lane, unsigned &cand, unsigned &c_hits) {
    constexpr bool K0 = (SH & kShK0) != 0;
    constexpr int NQ = QW / 4;
    LaneG2 g2;
    g2.x = pk2(B0.x[lane], B1.x[lane]); g2.y = pk2(B0.y[lane], B1.y[lane]); g2.z = pk2(B0.z[lane], B1.z[lane]);
    g2.sxx = pk2(B0.sxx[lane], B1.sxx[lane]); g2.syy = pk2(B0.syy[lane], B1.syy[lane]);
    g2.szz = pk2(B0.szz[lane], B1.szz[lane]); g2.sxy2 = pk2(B0.sxy2[lane], B1.sxy2[lane]);
    g2.sxz2 = pk2(B0.sxz2[lane], B1.sxz2[lane]); g2.syz2 = pk2(B0.syz2[lane], B1.syz2[lane]);
    if (n1 == 0) {  // the padding point in half 1
        float a, b;
        upk2(g2.x, a, b); g2.x = pk2(a, 1e18f);
        upk2(g2.y, a, b); g2.y = pk2(a, 1e18f);
        upk2(g2.z, a, b); g2.z = pk2(a, 1e18f);
        upk2(g2.sxx, a, b); g2.sxx = pk2(a, 0.f);
        upk2(g2.syy, a, b); g2.syy = pk2(a, 0.f);
        upk2(g2.szz, a, b); g2.szz = pk2(a, 0.f);
        upk2(g2.sxy2, a, b); g2.sxy2 = pk2(a, 0.f);
        upk2(g2.sxz2, a, b); g2.sxz2 = pk2(a, 0.f);
        upk2(g2.syz2, a, b); g2.syz2 = pk2(a, 0.f);
    }
    if constexpr (EX) {
        LaneG h0, h1;
        upk2(g2.sxx, h0.sxx, h1.sxx); upk2(g2.syy, h0.syy, h1.syy); upk2(g2.szz, h0.szz, h1.szz);
        upk2(g2.sxy2, h0.sxy2, h1.sxy2); upk2(g2.sxz2, h0.sxz2, h1.sxz2); upk2(g2.syz2, h0.syz2, h1.syz2);
        g2.f = pk2(half_tr_ss(h0), half_tr_ss(h1));
    }
    const unsigned nq = (unsigned)__popc(qm);
    c_hits += 4u * nq;
    cand += 4u * nq * (unsigned)(n0 + n1);
    const f32x2 nG2 = pk2(-k.G, -k.G), Gs2 = pk2(k.Gsmin, k.Gsmin);
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
        if (!((qm >> qq) & 1u)) continue;
        const int j0 = 4 * qq;
        f32x2 r2, sq;
        geom_g2<EX>(g2, wqd[j0], r2, sq);
        const f32x2 ir2 = reinterpret_cast<const ulonglong2 *>(&wqd[j0][1])->y;  // 1/r^2
        {
            // the quad's highest n_sigma copy first (see eval_chunk_pair)
            const f32x2 nmax = *reinterpret_cast<const f32x2 *>(&wqd[j0][2].z);  // -2 n_max
            float t0, t1;
            upk2(mul2(fma2(nmax, sq, r2), ir2), t0, t1);
            if (!__any_sync(0xffffffffu, t0 <= k.S_cut_u || t1 <= k.S_cut_u)) continue;
        }
#pragma unroll
        for (int j = j0; j < j0 + 4; ++j)
            tail_g2v<QW, K0>(A, j, r2, sq, ir2, *reinterpret_cast<const f32x2 *>(&wqd[j][2]), k, nG2, Gs2);
    }
}

// One stage of a kShQuad consumer warp: lane l tests quad l % NQ against
// slot base + l / NQ (one reach test per quad and staged chunk, the same test
// as the quad test of the general path; no warp-box test first), then the
// chunks some quad reaches are evaluated two at a time in slot order.
// Returns the number of slots some quad reaches.
template <int QW, bool EX, int SH, class C>
__device__ __forceinline__ int quad_stage(Acc<0, QW, 0, false> &A, EvalSmem<C> *sm, int s, int nslots, int warp,
                                          int lane, float4 (*wqd)[3], const QueryConsts &k, float pad_abs,
                                          unsigned &cand, unsigned &c_hits) {
    constexpr int NQ = QW / 4;
    constexpr int SPR = 32 / NQ;  // slots per round
    unsigned myq = 0u;            // lane t: the quads reaching slot t
#pragma unroll 1
    for (int base = 0; base < nslots; base += SPR) {
        const int sl = base + lane / NQ;
        bool qp = false;
        if (sl < nslots) qp = reaches<0, EX>(sm->wquad[warp][lane % NQ], sm->blk[s][sl].lo, sm->blk[s][sl].hi,
                                             pad_abs, k.S_reach);
        const unsigned hits = __ballot_sync(0xffffffffu, qp);
        const int r = lane - base;
        if (r >= 0 && r < SPR) myq = (hits >> (r * NQ)) & ((1u << NQ) - 1u);
    }
    unsigned cmask = __ballot_sync(0xffffffffu, myq != 0u);
    const int npass = __popc(cmask);
    while (cmask) {
        const int sa = __ffs(cmask) - 1;
        cmask &= cmask - 1;
        int sb = sa, n1 = 0;
        if (cmask) {
            sb = __ffs(cmask) - 1;
            cmask &= cmask - 1;
            n1 = sm->meta[s][sb].hi;
        }
        const unsigned qm = __shfl_sync(0xffffffffu, myq, sa) | __shfl_sync(0xffffffffu, myq, sb);
        eval_pair_quads<QW, EX, SH>(A, sm->blk[s][sa], sm->meta[s][sa].hi, sm->blk[s][sb], n1, qm, wqd, k, lane,
                                    cand, c_hits);
    }
    return npass;
}

// The adjoint counterpart of eval_chunk_pair (spheres, mean or sum cost).
template <int QW, int GROUP, bool FWD>
__device__ __forceinline__ void eval_chunk_pair_grad(Acc<0, QW, 0, true> &A, const ChunkBlock &B0,
                                                     const SlotMeta mt0, const ChunkBlock &B1, const SlotMeta mt1,
                                                     unsigned qmask, float4 (*wqd)[3], const QueryConsts &k,
                                                     int lane, unsigned &cand, unsigned &c_hits) {
    if (qmask == 0u) return;
    LaneG g0, g1;
    lane_gaussian(B0, mt0, lane, g0);
    lane_gaussian(B1, mt1, lane, g1);
    LaneG2 g2;
    g2.x = pk2(g0.x, g1.x); g2.y = pk2(g0.y, g1.y); g2.z = pk2(g0.z, g1.z);
    g2.sxx = pk2(g0.sxx, g1.sxx); g2.syy = pk2(g0.syy, g1.syy); g2.szz = pk2(g0.szz, g1.szz);
    g2.sxy2 = pk2(g0.sxy2, g1.sxy2); g2.sxz2 = pk2(g0.sxz2, g1.sxz2); g2.syz2 = pk2(g0.syz2, g1.syz2);
    unsigned gm = qmask;
#pragma unroll
    for (int sh = 1; sh < GROUP; sh <<= 1) gm |= gm >> sh;
    constexpr unsigned LEAD = GROUP == 1 ? 0xFFFFFFFFu : GROUP == 2 ? 0x55555555u : GROUP == 4 ? 0x11111111u
                                                                               : 0x01010101u;
    gm &= LEAD;
    const unsigned ng = (unsigned)__popc(gm) * (unsigned)GROUP;
    c_hits += ng;
    cand += ng * (unsigned)((mt0.hi - mt0.lo) + (mt1.hi - mt1.lo));
#pragma unroll
    for (int j0 = 0; j0 < QW; j0 += GROUP) {
        if ((gm >> j0) & 1u) {
#pragma unroll
            for (int j = j0; j < j0 + GROUP; ++j) pair_update_g2_grad<QW, FWD>(A, j, g2, wqd[j], k);
        }
    }
}

// One staged chunk against the primitives of `qmask`: lane l takes Gaussian
// l of the chunk (lanes outside the staged range hold a point that meets no
// primitive), then the primitives are evaluated two per basic block.
template <int PRIM, int QW, int MODE, bool GRAD, bool EX, bool FWD = false>
__device__ __forceinline__ void eval_chunk(Acc<PRIM, QW, MODE, GRAD> &A, const ChunkBlock &B, const SlotMeta &mt,
                                           unsigned qmask, float4 (*wq)[kQRec], const QueryConsts &k, int lane,
                                           int &group, unsigned &cand, unsigned &c_hits) {
    if (qmask == 0u) return;
    c_hits += (unsigned)__popc(qmask);
    if (MODE == 0 && !GRAD && PRIM == 1) {
        // fixed grouping of the cost partials (16 chunks) keeps the
        // summation order independent of the tile
        const int grp = mt.chunk >> 4;
        if (grp != group) {
#pragma unroll
            for (int j = 0; j < QW; ++j) { A.sum[j] += A.sumb[j]; A.sumb[j] = 0.f; }
            group = grp;
        }
    }
    LaneG g;
    lane_gaussian(B, mt, lane, g);
    g.f = 0.f;
    if constexpr (EX && PRIM == 0) g.f = half_tr_ss(g);
    cand += (unsigned)__popc(qmask) * (unsigned)(mt.hi - mt.lo);
    {
#pragma unroll
        for (int j = 0; j < QW; j += 2) {
            const bool p0 = (qmask >> j) & 1u, p1 = (qmask >> (j + 1)) & 1u;
            if (p0 && p1) {
                pair_update<PRIM, QW, MODE, GRAD, EX, FWD>(A, j, g, wq[j], k);
                pair_update<PRIM, QW, MODE, GRAD, EX, FWD>(A, j + 1, g, wq[j + 1], k);
            } else if (p0) {
                pair_update<PRIM, QW, MODE, GRAD, EX, FWD>(A, j, g, wq[j], k);
            } else if (p1) {
                pair_update<PRIM, QW, MODE, GRAD, EX, FWD>(A, j + 1, g, wq[j + 1], k);
            }
        }
    }
}

// kkp (persistent shapes): the stage sequence number, continued across tiles;
// the tile's terminator stage is released and *kkp advanced past it.
// Returns false when a bounded wait gave up.
template <int PRIM, class C, int MODE, bool GRAD, bool EX, int SH>
__device__ bool consumer_warp(const EvalArgs &a, EvalSmem<C> *sm, int tile, int warp, bool abort,
                              int *kkp = nullptr) {
    constexpr int RECS = PrimTraits<PRIM>::RECS;
    constexpr int QW = C::QW;
    constexpr int TQ = C::NCW * QW;
    const int lane = threadIdx.x & 31;
    const QueryConsts &k = a.k;
    const SceneDev &sc = a.sc;
    float4(*wq)[kQRec] = &sm->q[warp * QW];
    // ---- this warp's primitives into shared memory
    int nvalid = 0;
    if (lane < QW) {
        const int q = tile * TQ + C::row(warp, lane);
        float4 d0 = make_float4(0, 0, 0, 0), d1 = d0, d2 = d0, d3 = d0;
        if (q < a.Q) {
            const float4 *rec = row_rec<RECS>(a, q);
            const float4 r0 = rec[0];
            if (rec_valid(r0)) {
                const float ns = row_ns(a, q);
                float alpha, beta;
                prim_reach<PRIM, EX>(rec, ns, k.S_reach, alpha, beta);
                if (PRIM == 0) {
                    d0 = make_float4(r0.x, r0.y, r0.z, 1.f / (r0.w * r0.w));
                    d1 = make_float4(2.f * ns, alpha, beta, 1.f);
                } else {
                    const float4 r1 = rec[1], r2 = rec[2];
                    d0 = make_float4(r0.x, r0.y, r0.z, 2.f * ns);
                    d1 = r1;
                    d2 = make_float4(r2.x, r2.y, alpha, beta);
                    d3 = make_float4(1.f, 1.f / r2.z, 0.f, 0.f);
                }
                nvalid = 1;
            }
        }
        wq[lane][0] = d0;
        wq[lane][1] = d1;
        wq[lane][2] = d2;
        wq[lane][3] = d3;
    }
    constexpr unsigned QBITS = (1u << QW) - 1u;
    const unsigned wvalid = __ballot_sync(0xffffffffu, nvalid != 0) & QBITS;  // bit j: primitive j is valid
    nvalid = __reduce_add_sync(0xffffffffu, nvalid);
    // flags mode: primitives still open (bit j), those settled by their group,
    // and lane j's group index (-1: no group)
    unsigned wlive = wvalid, wgset = 0u;
    int mygrp = -1;
    if (MODE == 3 && a.gflags && k.group_size > 0 && lane < QW && ((wvalid >> lane) & 1u)) {
        const int q = tile * TQ + C::row(warp, lane);
        mygrp = (int)(row_out(a, q) / (uint32_t)k.group_size);
        if (!CS_IDX_OK(mygrp < (a.Q + k.group_size - 1) / k.group_size, a.err)) mygrp = -1;
    }
    if (MODE == 3 && wlive == 0u && lane == 0) atomicSub(&sm->active, 1);
    __syncwarp();
    float4(*wqd)[3] = &sm->qd[warp * QW];
    if (PRIM == 0 && lane < QW) {
        const float4 a = wq[lane][0], b = wq[lane][1];
        wqd[lane][0] = make_float4(-a.x, -a.x, -a.y, -a.y);
        wqd[lane][1] = make_float4(-a.z, -a.z, a.w, a.w);
        wqd[lane][2] = make_float4(-b.x, -b.x, 0.f, 0.f);
    }
    __syncwarp();
    if ((SH & kShGeom) && PRIM == 0 && lane < QW && (lane & 3) == 0) {
        // row quads of a sweep: -2 n_max of rows lane .. lane + 3 beside row lane's -2 n
        // (read only when the four rows are one sphere)
        float m = wqd[lane][2].x;
#pragma unroll
        for (int r = 1; r < 4; ++r) m = fminf(m, wqd[lane + r][2].x);
        wqd[lane][2].z = m;
        wqd[lane][2].w = m;
    }
    __syncwarp();
    // same, bit j (j even): rows j and j + 1 are the same sphere (centre and
    // radius bit for bit, both valid), so the packed evaluation shares their
    // geometry; link, bit j (j even, j > 0): rows j - 1 and j are too
    unsigned same = 0u, link = 0u;
    if ((SH & kShGeom) && PRIM == 0) {
        bool eq = false;
        if (lane < QW - 1) {
            const float4 a = wq[lane][0], b = wq[lane + 1][0];
            eq = ((wvalid >> lane) & 3u) == 3u && __float_as_uint(a.x) == __float_as_uint(b.x) &&
                 __float_as_uint(a.y) == __float_as_uint(b.y) && __float_as_uint(a.z) == __float_as_uint(b.z) &&
                 __float_as_uint(a.w) == __float_as_uint(b.w);
        }
        const unsigned e = __ballot_sync(0xffffffffu, eq);
        same = e & 0x55555555u;
        link = (e & 0xAAAAAAAAu) << 1;
    }
    // Quads of a sweep evaluated as groups of four: when every quad of the
    // warp is one sphere, one reach test per quad replaces the four row
    // tests.  The test takes the largest alpha and beta of the quad's rows,
    // so it reaches at least as far as each row; a row that does not reach a
    // chunk adds nothing, so the outputs do not change.
    constexpr bool QT = (SH & kShGeom) && PRIM == 0 && C::GROUP == 4 && C::IL == 4 && MODE == 0 && !GRAD;
    constexpr int NQ = QW / 4;  // quads per warp
    bool quadok = false;
    if constexpr (QT) {
        if (lane < NQ) {  // quad `lane` as one record
            float4 r0 = wq[4 * lane][0], r1 = wq[4 * lane][1];
#pragma unroll
            for (int m = 1; m < 4; ++m) {
                const float4 b = wq[4 * lane + m][1];
                r1.y = fmaxf(r1.y, b.y);
                r1.z = fmaxf(r1.z, b.z);
                r1.w = fmaxf(r1.w, b.w);
            }
            sm->wquad[warp][lane][0] = r0;
            sm->wquad[warp][lane][1] = r1;
        }
        unsigned whole = 0u;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq)
            whole |= ((same >> (4 * qq)) & (same >> (4 * qq + 2)) & (link >> (4 * qq + 2)) & 1u) << qq;
        quadok = whole == (1u << NQ) - 1u;
    }
    // the warp's box of primitive centres and its largest reach parameters:
    // a chunk outside box + reach is out of reach of every primitive here
    // (the whole-quad sweep path tests its quads directly and needs none)
    if constexpr (!(QT && (SH & kShQuad) != 0)) {
        float wlx = INFINITY, wly = INFINITY, wlz = INFINITY, whx = -INFINITY, why = -INFINITY, whz = -INFINITY;
        float wal = 0.f, wbe = 0.f;
        if (lane < QW) {
            const float4 q0 = wq[lane][0];
            float alpha, beta, live;
            if (PRIM == 0) { const float4 q1 = wq[lane][1]; alpha = q1.y; beta = q1.z; live = q1.w; }
            else { const float4 q2 = wq[lane][2]; alpha = q2.z; beta = q2.w; live = wq[lane][3].x; }
            if (live != 0.f) {
                wlx = whx = q0.x; wly = why = q0.y; wlz = whz = q0.z;
                wal = alpha; wbe = beta;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            wlx = fminf(wlx, __shfl_xor_sync(0xffffffffu, wlx, o));
            wly = fminf(wly, __shfl_xor_sync(0xffffffffu, wly, o));
            wlz = fminf(wlz, __shfl_xor_sync(0xffffffffu, wlz, o));
            whx = fmaxf(whx, __shfl_xor_sync(0xffffffffu, whx, o));
            why = fmaxf(why, __shfl_xor_sync(0xffffffffu, why, o));
            whz = fmaxf(whz, __shfl_xor_sync(0xffffffffu, whz, o));
            wal = fmaxf(wal, __shfl_xor_sync(0xffffffffu, wal, o));
            wbe = fmaxf(wbe, __shfl_xor_sync(0xffffffffu, wbe, o));
        }
        if (lane == 0) {
            sm->wbox[warp][0] = make_float4(wlx, wly, wlz, wal);
            sm->wbox[warp][1] = make_float4(whx, why, whz, wbe);
        }
        __syncwarp();
    }
    Acc<PRIM, QW, MODE, GRAD> A;
    A.fin = 0u;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
        if constexpr (MODE != 3) A.cnt[j] = 0;
        constexpr bool FWD = (SH & kShFwd) != 0;
        if (!GRAD || FWD) A.cin[j] = 0;
        if (MODE == 0 && (!GRAD || FWD)) { A.sum[j] = 0.f; if (PRIM == 1) A.sumb[j] = 0.f; }

        if (MODE == 1) A.mn[j] = INFINITY;
        if (MODE == 2) { A.sm_m[j] = k.S_cut; A.sm_acc[j] = 0.f; }
        if (GRAD) { A.gx[j] = 0.f; A.gy[j] = 0.f; A.gz[j] = 0.f; }
    }
    unsigned cand = 0, c_hits = 0;  // (primitive, Gaussian) pairs and (primitive, chunk) hits evaluated
    unsigned long long *wst = sm->wst[warp];
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < 6; ++i) wst[i] = 0ull;
        wst[6] = (unsigned long long)clock64();
    }
    int group = -1;               // chunk group of the cost partials
    bool ok = !abort;
    for (int kk = kkp ? *kkp : 0; ok; ++kk) {
        const int s = kk % C::NS;
        bool got = true;
        if (lane == 0) {
            const long long c0 = clock64();
            const long long w = wait_phase(&sm->full[s], (unsigned)((kk / C::NS) & 1), a.wait_polls);
            const long long c1 = clock64();
            wst[4] += (unsigned long long)(c1 - c0);
            if (kk == 0) wst[5] = (unsigned long long)c1 - wst[6];
            got = w >= 0;
            wst[3] += got ? (unsigned long long)w : 0ull;
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        const int nslots = sm->count[s];
        if (nslots == 0) {
            if (kkp) {  // release the terminator: the ring runs on into the next tile
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->empty[s]);
                *kkp = kk + 1;
            }
            break;
        }
        if (lane == 0) {
            wst[0] += 1ull;
            wst[1] += (unsigned long long)nslots;
        }
        if constexpr (MODE == 3) {
            // settle primitives whose in-count already exceeds k_thr (their
            // flag cannot change) or whose group already collides
            if (wlive) {
                unsigned still = wlive;
#pragma unroll
                for (int j = 0; j < QW; ++j) {
                    if ((wlive >> j) & 1u) {
                        const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)A.cin[j]);
                        const int g = __shfl_sync(0xffffffffu, mygrp, j);
                        const bool own = tot > k.k_thr;
                        bool grp = false;
                        if (own) {
                            if (lane == 0 && g >= 0) atomicOr(&a.gflags[g], 1u);
                        } else if (g >= 0) {
                            grp = __shfl_sync(0xffffffffu, *(volatile unsigned *)&a.gflags[g] != 0u, 0);
                        }
                        if (own || grp) still &= ~(1u << j);
                        if (grp) wgset |= 1u << j;
                    }
                }
                if (still != wlive) {
                    if (lane < QW && (((wlive & ~still) >> lane) & 1u)) {
                        if (PRIM == 0) wq[lane][1].w = 0.f;  // the live flag the reach tests read
                        else wq[lane][3].x = 0.f;
                    }
                    __syncwarp();
                    wlive = still;
                    if (wlive == 0u && lane == 0) atomicSub(&sm->active, 1);
                }
            }
        }
        if constexpr (QT && (SH & kShQuad) != 0) {
            if (nvalid > 0) {
                const int npass = quad_stage<QW, EX, SH>(A, sm, s, nslots, warp, lane, wqd, k, sc.pad_abs, cand, c_hits);
                if (lane == 0) wst[2] += (unsigned long long)npass;
            }
        } else if ((MODE == 3) ? (wlive != 0u) : (nvalid > 0)) {
            // lane t tests chunk slot t against the warp's box + reach
            bool wpass = false;
            if (lane < nslots) {
                const float4 blo = sm->blk[s][lane].lo, bhi = sm->blk[s][lane].hi;
                const float4 wl = sm->wbox[warp][0], wh = sm->wbox[warp][1];
                const float R = reach<EX && PRIM == 0>(wl.w, wh.w, blo.w, sc.pad_abs);
                wpass = box_gap2(wl.x, wl.y, wl.z, wh.x, wh.y, wh.z, blo, bhi) <= R * R;
            }
            unsigned pmask = __ballot_sync(0xffffffffu, wpass);
            if (lane == 0) wst[2] += (unsigned long long)__popc(pmask);
            // then (primitive, chunk) tests, 32 / QW chunks per round (lane l:
            // primitive l % QW, chunk l / QW of the round); myq of lane t
            // collects slot t's mask of the primitives that reach it
            constexpr int CPR = 32 / QW;
            constexpr unsigned QMASK = (1u << QW) - 1u;
            unsigned myq = 0u;
            if (QT && (quadok || (SH & kShQuad))) {
                // lane l: quad l % NQ against the passing slot of rank
                // base + l / NQ; slot t's quad bits become its row bits
                constexpr int CPRQ = 32 / NQ;
                const int rank = __popc(pmask & ((1u << lane) - 1u));
                const bool mine = (pmask >> lane) & 1u;
                const int npass = __popc(pmask);
                if (mine) sm->slots[warp][rank] = lane;
                __syncwarp();
                for (int base = 0; base < npass; base += CPRQ) {
                    const int kq = base + lane / NQ;
                    bool qp = false;
                    if (kq < npass) {
                        const int my = sm->slots[warp][kq];
                        qp = reaches<0, EX>(sm->wquad[warp][lane % NQ], sm->blk[s][my].lo, sm->blk[s][my].hi,
                                            sc.pad_abs, k.S_reach);
                    }
                    const unsigned hits = __ballot_sync(0xffffffffu, qp);
                    if (mine && rank >= base && rank < base + CPRQ) {
                        const unsigned qb = hits >> ((rank - base) * NQ);
#pragma unroll
                        for (int qq = 0; qq < NQ; ++qq) myq |= ((qb >> qq) & 1u) ? 0xFu << (4 * qq) : 0u;
                    }
                }
                __syncwarp();  // every lane has read the list before the next stage rewrites it
                pmask = 0u;
            }
            while (pmask) {
                int sl[CPR];
#pragma unroll
                for (int r = 0; r < CPR; ++r) {
                    sl[r] = pmask ? __ffs(pmask) - 1 : -1;
                    pmask &= pmask - 1;
                }
                const int part = lane / QW;
                int my = sl[0];
#pragma unroll
                for (int r = 1; r < CPR; ++r) my = part == r ? sl[r] : my;
                bool qp = false;
                if (my >= 0) qp = reaches<PRIM, EX>(wq[lane % QW], sm->blk[s][my].lo, sm->blk[s][my].hi, sc.pad_abs, k.S_reach);
                const unsigned hits = __ballot_sync(0xffffffffu, qp);
#pragma unroll
                for (int r = 0; r < CPR; ++r)
                    if (lane == sl[r]) myq = (hits >> (r * QW)) & QMASK;
            }
            unsigned cmask = __ballot_sync(0xffffffffu, myq != 0u);
            if constexpr (PRIM == 0 && MODE == 0 && !GRAD) {
                // spheres, cost reductions: chunks with hits in pairs, two
                // Gaussians per lane in packed registers
                while (cmask) {
                    const int sa = __ffs(cmask) - 1;
                    cmask &= cmask - 1;
                    int sb = -1;
                    if (cmask) {
                        sb = __ffs(cmask) - 1;
                        cmask &= cmask - 1;
                    }
                    const unsigned qa = __shfl_sync(0xffffffffu, myq, sa);
                    const unsigned qb = sb >= 0 ? __shfl_sync(0xffffffffu, myq, sb) : 0u;
                    eval_chunk_pair<QW, C::GROUP, EX, SH, C::QUAD>(A, sm->blk[s][sa], sm->meta[s][sa], sm->blk[s][sb >= 0 ? sb : sa],
                                                  sb >= 0 ? sm->meta[s][sb] : SlotMeta{0, 0, 0, 0}, qa | qb, wqd, k,
                                                  lane, cand, c_hits, same, link);
                }
            } else if constexpr (PRIM == 0 && MODE == 0 && GRAD && !EX) {
                // the sphere cost adjoint: the same chunk pairs in packed registers
                while (cmask) {
                    const int sa = __ffs(cmask) - 1;
                    cmask &= cmask - 1;
                    int sb = -1;
                    if (cmask) {
                        sb = __ffs(cmask) - 1;
                        cmask &= cmask - 1;
                    }
                    const unsigned qa = __shfl_sync(0xffffffffu, myq, sa);
                    const unsigned qb = sb >= 0 ? __shfl_sync(0xffffffffu, myq, sb) : 0u;
                    eval_chunk_pair_grad<QW, C::GROUP, (SH & kShFwd) != 0>(
                        A, sm->blk[s][sa], sm->meta[s][sa], sm->blk[s][sb >= 0 ? sb : sa],
                        sb >= 0 ? sm->meta[s][sb] : SlotMeta{0, 0, 0, 0}, qa | qb, wqd, k, lane, cand, c_hits);
                }
            } else {
#pragma unroll 1
                while (cmask) {
                    const int sl = __ffs(cmask) - 1;
                    cmask &= cmask - 1;
                    const unsigned q = __shfl_sync(0xffffffffu, myq, sl);
                    eval_chunk<PRIM, QW, MODE, GRAD, EX, (SH & kShFwd) != 0>(A, sm->blk[s][sl], sm->meta[s][sl], q, wq, k, lane, group,
                                                         cand, c_hits);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm->empty[s]);
    }
    if (!ok && !abort && lane == 0) atomicOr(a.err, kErrTimeout);
    const unsigned long long c_loop_end = (unsigned long long)clock64();

    // ---- reductions across lanes (fixed trees) and outputs
    // Each row's reductions run over the warp (fixed trees, the results on
    // every lane); lane j keeps row j's results and, after the loop, the
    // first QW lanes write their rows' outputs at once (output row, upstream
    // gradient and the divisions computed per lane in parallel rather than
    // one row after another).
    const bool mine = lane < QW;
    const int my_q = tile * TQ + C::row(warp, mine ? lane : 0);
    const bool my_in = mine && my_q < a.Q;
    const bool my_good = my_in && ((wvalid >> lane) & 1u) && ok;
    float my_tot = 0.f, my_gx = 0.f, my_gy = 0.f, my_gz = 0.f, my_f = 0.f;
    int my_cnt = 0, my_cin = 0;
    unsigned long long nb_total = 0;
#pragma unroll
    for (int j = 0; j < QW; ++j) {
        const bool vq = (wvalid >> j) & 1u;
        if constexpr (MODE == 3) {
            // 1: in collision; 0: free; 2: not finished because its group collides
            const int cinj = (int)__reduce_add_sync(0xffffffffu, (unsigned)A.cin[j]);
            if (lane == j) my_cin = cinj > k.k_thr ? 1 : ((wgset >> j) & 1u) ? 2 : 0;
            continue;
        } else {
        const int cntj = __reduce_add_sync(0xffffffffu, (unsigned)A.cnt[j]);
        if (!GRAD) {
            int cinj;
            if constexpr ((SH & kShK0) && PRIM == 0 && MODE == 0) {
                cinj = __any_sync(0xffffffffu, (A.fin >> j) & 1u) ? 1 : 0;  // k_thr = 0: any pair in collision
            } else {
                cinj = (int)__reduce_add_sync(0xffffffffu, (unsigned)A.cin[j]);
            }
            float metric = 0.f;  // mode 0: the sum, scaled after the loop
            if (MODE == 0) {
                metric = warp_sum(PRIM == 1 ? A.sum[j] + A.sumb[j] : A.sum[j]);
            } else if (MODE == 1) {
                const float m = warp_min(A.mn[j]);
                metric = cntj > 0 ? m : INFINITY;
            } else {
                const float M = warp_min(A.sm_m[j]);
                const float acc = warp_sum(A.sm_acc[j] * ex2_approx((M - A.sm_m[j]) * k.K));
                metric = cntj > 0 ? M - k.tau * 0.6931471805599453f * lg2_approx(acc) : INFINITY;
            }
            if (lane == j) { my_tot = metric; my_cnt = cntj; my_cin = cinj; }
        } else {
            float gx, gy, gz, f = 0.f;
            if (MODE == 0) {
                gx = warp_sum(A.gx[j]); gy = warp_sum(A.gy[j]); gz = warp_sum(A.gz[j]);
            } else if (MODE == 1) {
                // the arg-min pair: the lane holding the smallest st2 (lowest lane on ties)
                const float m = warp_min(A.mn[j]);
                const unsigned who = __ballot_sync(0xffffffffu, A.mn[j] == m);
                const int src = who ? __ffs(who) - 1 : 0;
                gx = __shfl_sync(0xffffffffu, A.gx[j], src);
                gy = __shfl_sync(0xffffffffu, A.gy[j], src);
                gz = __shfl_sync(0xffffffffu, A.gz[j], src);
                f = cntj > 0 ? 1.f : 0.f;
            } else {
                const float M = warp_min(A.sm_m[j]);
                const float sc_ = ex2_approx((M - A.sm_m[j]) * k.K);
                const float acc = warp_sum(A.sm_acc[j] * sc_);
                gx = warp_sum(A.gx[j] * sc_); gy = warp_sum(A.gy[j] * sc_); gz = warp_sum(A.gz[j] * sc_);
                f = cntj > 0 ? 1.f / acc : 0.f;
            }
            if (lane == j) { my_gx = gx; my_gy = gy; my_gz = gz; my_f = f; my_cnt = cntj; }
            if constexpr ((SH & kShFwd) != 0 && MODE == 0 && PRIM == 0) {
                // the forward outputs of the same launch (as in the forward epilogue)
                const int cinj = (int)__reduce_add_sync(0xffffffffu, (unsigned)A.cin[j]);
                const float tot = warp_sum(A.sum[j]);
                if (lane == j) { my_tot = tot; my_cin = cinj; }
            }
        }
        if (vq) nb_total += (unsigned long long)cntj;
        }  // MODE != 3
    }
    if (my_in) {
        const uint32_t row = row_out(a, my_q);
        const float nanv = __int_as_float(0x7fc00000);
        if constexpr (MODE == 3) {
            if (a.out_collide) a.out_collide[row] = my_good ? (uint8_t)my_cin : (uint8_t)0;
        } else if constexpr (!GRAD) {
            float metric = my_tot;
            if (MODE == 0)
                metric = (k.mode == CS_METRIC_MEAN_COST) ? (my_cnt > 0 ? my_tot * k.d_max / (float)my_cnt : 0.f)
                                                         : my_tot * k.d_max;
            if (a.out_metric) a.out_metric[row] = my_good ? metric : nanv;
            if (a.out_collide) a.out_collide[row] = (my_good && my_cin > k.k_thr) ? 1 : 0;
            if (a.out_count) a.out_count[row] = my_good ? my_cnt : 0;
        } else {
            float f = my_f;
            if (MODE == 0)
                f = (k.mode == CS_METRIC_MEAN_COST) ? (my_cnt > 0 ? -k.gamma * k.d_max / (float)my_cnt : 0.f)
                                                    : -k.gamma * k.d_max;
            if constexpr ((SH & kShFwd) != 0 && MODE == 0 && PRIM == 0) {
                const float metric = (k.mode == CS_METRIC_MEAN_COST)
                                         ? (my_cnt > 0 ? my_tot * k.d_max / (float)my_cnt : 0.f)
                                         : my_tot * k.d_max;
                if (a.out_metric) a.out_metric[row] = my_good ? metric : nanv;
                if (a.out_collide) a.out_collide[row] = (my_good && my_cin > k.k_thr) ? 1 : 0;
                if (a.out_count) a.out_count[row] = my_good ? my_cnt : 0;
            }
            float up = 1.f;
            if (a.grad_out) {
                const uint32_t gi = k.group_size > 0 ? row / (uint32_t)k.group_size : row;
                up = a.grad_out[CS_IDX_OK(gi < (uint32_t)a.Q, a.err) ? gi : 0u];
            }
            a.grad_centres[3 * (size_t)row + 0] = my_good ? my_gx * f * up : nanv;
            a.grad_centres[3 * (size_t)row + 1] = my_good ? my_gy * f * up : nanv;
            a.grad_centres[3 * (size_t)row + 2] = my_good ? my_gz * f * up : nanv;
        }
    }
    if (a.stats && lane == 0) {
        atomicAdd(a.stats + 0, (unsigned long long)cand);
        atomicAdd(a.stats + 1, nb_total);
    }
    if (a.kstats && lane == 0) {
        atomicAdd(a.kstats + 0, wst[0]);
        atomicAdd(a.kstats + 1, wst[1]);
        atomicAdd(a.kstats + 2, wst[2]);
        atomicAdd(a.kstats + 3, (unsigned long long)c_hits);
        atomicAdd(a.kstats + 6, wst[3]);
        const unsigned long long c_end = (unsigned long long)clock64();
        atomicAdd(a.kstats + 8, c_end - wst[6]);
        atomicAdd(a.kstats + 9, wst[4]);
        atomicAdd(a.kstats + 12, wst[5]);
        atomicAdd(a.kstats + 14, c_end - c_loop_end);
    }
    return ok;
}

template <int PRIM, class C, int MODE, bool GRAD, bool EX = false, int SH = 0>
__global__ void __launch_bounds__((C::NCW + 1) * 32, C::MINB) k_eval(const EvalArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    EvalSmem<C> *sm = reinterpret_cast<EvalSmem<C> *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::NS; ++s) {
            mbar_init(&sm->full[s], 1);
            mbar_init(&sm->empty[s], C::NCW);
        }
        if (C::PERSIST) {
            for (int s = 0; s < 2; ++s) {
                mbar_init(&sm->tfull[s], 1);
                mbar_init(&sm->tempty[s], C::NCW);
            }
        }
        fence_mbar_init();
        sm->abort = (*(volatile unsigned *)a.err & kErrTimeout) ? 1 : 0;
        sm->active = C::NCW;
    }
    __syncthreads();
    const bool abort = sm->abort != 0;
    if constexpr (C::PERSIST) {
        static_assert(MODE != 3, "the flags mode's early exit runs one tile per CTA");
        const int lane = threadIdx.x & 31;
        if (warp == C::NCW) {
            if (!abort) producer_persistent<PRIM, C, EX>(a, sm);
        } else if (abort) {
            // an earlier launch on this stream timed out: mark every row as
            // the one-tile-per-CTA shapes do (NaN metric and gradient, flag and
            // count 0), with no waits
            for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x)
                if (lane < C::QW) {
                    const int q = t * C::NCW * C::QW + C::row(warp, lane);
                    if (q < a.Q) {
                        const uint32_t row = row_out(a, q);
                        const float nanv = __int_as_float(0x7fc00000);
                        if (a.out_metric) a.out_metric[row] = nanv;
                        if (a.out_collide) a.out_collide[row] = 0;
                        if (a.out_count) a.out_count[row] = 0;
                        if (GRAD && a.grad_centres) {
                            a.grad_centres[3 * (size_t)row + 0] = nanv;
                            a.grad_centres[3 * (size_t)row + 1] = nanv;
                            a.grad_centres[3 * (size_t)row + 2] = nanv;
                        }
                    }
                }
        } else {
            int kk = 0;
            for (int i = 0;; ++i) {
                const int slot = i & 1;
                bool got = true;
                if (lane == 0) got = wait_phase(&sm->tfull[slot], (unsigned)((i >> 1) & 1), a.wait_polls) >= 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                const int t = got ? *(volatile int *)&sm->tile_q[slot] : -1;
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm->tempty[slot]);
                if (!got && lane == 0) atomicOr(a.err, kErrTimeout);
                if (t < 0 || t >= a.ntiles) break;
                if (!consumer_warp<PRIM, C, MODE, GRAD, EX, SH>(a, sm, t, warp, false, &kk)) break;
            }
        }
    } else {
        const int tile = blockIdx.x;
        if (warp == C::NCW) {
            if (!abort) producer_warp<PRIM, C, EX>(a, sm, tile, MODE == 3);
        } else {
            consumer_warp<PRIM, C, MODE, GRAD, EX, SH>(a, sm, tile, warp, abort);
        }
    }
}

// ------------------------------------------------------ preparation kernels
constexpr int kBucketBits = 16;            // buckets of the small-batch counting sort
constexpr int kBucketShift = 29 - kBucketBits;  // keys have 29 bits (24 Morton + 5 size class)
constexpr int kBucketMaxQ = 1 << 17;       // batches up to this size take the counting sort
constexpr uint32_t kBuckets() { return 1u << kBucketBits; }
__device__ __forceinline__ uint32_t spread8(uint32_t v) {
    v &= 0xFFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Sort key of each primitive: the Morton code of its centre over the scene
// box (8 bits per axis) above its size class (half-octaves of the radius or
// largest semi-axis, from 1/1024 up).  Tiles of consecutive keys then hold
// primitives close together, so the tile box the producer culls with stays
// small even when a batch is sparse and mixes many sizes.
__global__ void k_prep_keys(const float *__restrict__ prims, int prim_type, int Q, SceneDev sc,
                            uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                            uint32_t *__restrict__ bucket_hist) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Q) return;
    const int stride = prim_type == CS_PRIM_SPHERE ? 4 : 10;
    const float *p = prims + (size_t)j * stride;
    uint32_t c[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float u = (p[a] - sc.bb_lo[a]) / (sc.bb_hi[a] - sc.bb_lo[a]) * 256.f;
        u = isfinite(u) ? fminf(fmaxf(u, 0.f), 255.f) : 255.f;
        c[a] = (uint32_t)u;
    }
    const uint32_t code = spread8(c[0]) | (spread8(c[1]) << 1) | (spread8(c[2]) << 2);
    const float size = prim_type == CS_PRIM_SPHERE ? p[3] : fmaxf(fmaxf(p[7], p[8]), p[9]);
    uint32_t cls = 31;
    if (size > 0.f && isfinite(size)) {
        const int bits = __float_as_int(size);
        const int half_oct = 2 * ((bits >> 23) & 0xFF) + ((bits >> 22) & 1) - 2 * (127 - 10);
        cls = (uint32_t)min(max(half_oct, 0), 31);
    }
    const uint32_t key = (code << 5) | cls;
    keys[j] = key;
    vals[j] = (uint32_t)j;
    if (bucket_hist) atomicAdd(&bucket_hist[key >> kBucketShift], 1u);
}

// Counting sort of the rows by the bucket of their key (the top 16 Morton
// bits: cells of 1/40 of the scene box per axis), for batches small enough
// that the key's full radix sort is launch-bound.  The order inside a bucket
// follows the atomics; that changes which rows share a tile, never a row's
// result (each row's reductions run in a fixed order whatever its tile).
// Warp-aggregated: lanes with the same bucket take one atomic.
__global__ void k_bucket_scatter(const uint32_t *__restrict__ keys, int Q, uint32_t *__restrict__ offs,
                                 uint32_t *__restrict__ perm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned active = __ballot_sync(0xffffffffu, j < Q);
    if (j >= Q) return;
    const uint32_t b = keys[j] >> kBucketShift;
    const unsigned peers = __match_any_sync(active, b);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&offs[b], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    perm[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)j;
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

// Section II-D/E group outputs: metric summed, flag OR-ed over runs of G rows
// (a warp per group from kGroupWarpMin rows, else a thread per group).
__global__ void k_group(const float *__restrict__ metric, const uint8_t *__restrict__ collide,
                        int Q, int G, float *__restrict__ gm, uint8_t *__restrict__ gc, unsigned *err) {
    const int ng = (Q + G - 1) / G;
    float sum;
    unsigned c;
    if (G >= kGroupWarpMin) {
        const int g = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
        if (g >= ng) return;  // whole warps leave together
        const int b = g * G, e = min(Q, b + G);
        if (kDebugBuild && err && !CS_IDX_OK(b >= 0 && b < e && e <= Q, err)) return;
        group_rows_warp(metric, collide, b, e, threadIdx.x & 31, sum, c);
        if ((threadIdx.x & 31) != 0) return;
        if (gm) gm[g] = sum;
        if (gc) gc[g] = (uint8_t)c;
    } else {
        const int g = blockIdx.x * blockDim.x + threadIdx.x;
        if (g >= ng) return;
        const int b = g * G, e = min(Q, b + G);
        if (kDebugBuild && err && !CS_IDX_OK(b >= 0 && b < e && e <= Q, err)) return;
        group_rows_serial(metric, collide, b, e, sum, c);
        if (gm) gm[g] = sum;
        if (gc) gc[g] = (uint8_t)c;
    }
}

// ---------------------------------------------------------- host launchers
QueryConsts make_consts(const cs_params &p) {
    QueryConsts k;
    const double S_cut = (double)p.s_min + log(1.0 / (double)p.eps) / (double)p.gamma;
    k.S_cut = (float)S_cut;
    k.S_reach = (float)std::max(S_cut, 1.0);
    k.T_in = S_cut >= 1.0 ? 1.f : nextafterf(k.S_cut, INFINITY);
    k.S_cut_u = k.S_cut >= 0.f ? k.S_cut : -INFINITY;
    k.T_in_u = k.T_in > 0.f ? k.T_in : -INFINITY;
    k.G = (float)((double)p.gamma * 1.4426950408889634);
    k.Gsmin = (float)((double)p.gamma * 1.4426950408889634 * (double)p.s_min);
    k.E_cap = std::min(k.Gsmin, 0.f);
    k.s_min = p.s_min;
    k.d_max = p.d_max;
    k.gamma = p.gamma;
    k.tau = p.tau;
    k.K = (float)(1.0 / ((double)p.tau * 0.6931471805599453));
    k.k_thr = p.k_thr;
    k.mode = p.mode;
    k.group_size = p.group_size;
    k.exact = p.exact_variance;
    k.sweep = sweep_blocks(p);
    return k;
}


// Tile shapes (cs_tile_configs):
//   1: 8 consumer warps x 8 primitives, 4 stages x 16 chunks, 2 CTAs/SM (default)
//   2: 8 x 16, 4 x 16, 1 CTA/SM
//   3: 4 x 8, 3 x 8, 4 CTAs/SM
//   4: 4 x 16, 3 x 8, 3 CTAs/SM
//   5-8: shapes 1, 1, 4, 4 evaluating sphere primitives in groups of 4, 8, 4, 8
//   9: 8 x 8, 8 stages x 8 chunks, 2 CTAs/SM (deeper ring, same staging memory as 1)
//   10: 8 x 8, 16 stages x 4 chunks, 2 CTAs/SM
//   11: 4 x 16, 6 stages x 8 chunks, 3 CTAs/SM
//   12: shape 9 with groups of 4
//   13: 4 x 16, 3 stages x 16 chunks, 3 CTAs/SM
//   14: 4 x 16, 4 stages x 12 chunks, 3 CTAs/SM
//   15: 8 x 8, 2 stages x 32 chunks, 2 CTAs/SM
//   16: shape 1 with the tile's rows interleaved over the consumer warps
//   17-19: shapes 1, 15, 13 with row pairs interleaved over the consumer warps
//   20, 21: shape 18 evaluating sphere primitives one at a time / in groups of 4
//   22: 2 x 8, 2 stages x 12 chunks, 6 CTAs/SM (small or sparse batches: more, tighter tiles)
//   23: 1 x 8, 2 stages x 10 chunks, 8 CTAs/SM
//   24: shape 18 with row quads interleaved over the consumer warps (a
//       sweep's four n_sigma copies of a sphere in one warp)
//   25: shape 24 evaluating sphere primitives in groups of 4 (a quad)
//   26: shape 19 with row quads evaluated in groups of 4
//   27: 4 x 16, 2 stages x 24 chunks, 3 CTAs/SM, row quads in groups of 4
//   28: shape 27 as a persistent kernel (SMs x 3 CTAs taking tiles from a
//       counter; the producer stages the next tile while the consumers end
//       the current one); the flags mode runs its own shapes
//   29: 4 x 16, 2 stages x 16 chunks, 4 CTAs/SM, row quads in groups of 4
//       (at most 96 registers: the warp box and quad records live in shared
//       memory; four CTAs of five warps fill the register file)
//   30: shape 29 as a persistent kernel
using Cfg1 = Cfg<8, 8, 4, 16, 2>;
using Cfg2 = Cfg<8, 16, 4, 16, 1>;
using Cfg3 = Cfg<4, 8, 3, 8, 4>;
using Cfg4 = Cfg<4, 16, 3, 8, 3>;
using Cfg5 = Cfg<8, 8, 4, 16, 2, 4>;
using Cfg6 = Cfg<8, 8, 4, 16, 2, 8>;
using Cfg7 = Cfg<4, 16, 3, 8, 3, 4>;
using Cfg8 = Cfg<4, 16, 3, 8, 3, 8>;
using Cfg9 = Cfg<8, 8, 8, 8, 2>;
using Cfg10 = Cfg<8, 8, 16, 4, 2>;
using Cfg11 = Cfg<4, 16, 6, 8, 3>;
using Cfg12 = Cfg<8, 8, 8, 8, 2, 4>;
using Cfg13 = Cfg<4, 16, 3, 16, 3>;
using Cfg14 = Cfg<4, 16, 4, 12, 3>;
using Cfg15 = Cfg<8, 8, 2, 32, 2>;
using Cfg16 = Cfg<8, 8, 4, 16, 2, 2, 1>;
using Cfg17 = Cfg<8, 8, 4, 16, 2, 2, 2>;
using Cfg18 = Cfg<8, 8, 2, 32, 2, 2, 2>;
using Cfg19 = Cfg<4, 16, 3, 16, 3, 2, 2>;
using Cfg20 = Cfg<8, 8, 2, 32, 2, 1, 2>;
using Cfg21 = Cfg<8, 8, 2, 32, 2, 4, 2>;
using Cfg22 = Cfg<2, 8, 2, 12, 6, 2, 2>;
using Cfg23 = Cfg<1, 8, 2, 10, 8, 2, 0>;
using Cfg24 = Cfg<8, 8, 2, 32, 2, 2, 4>;
using Cfg25 = Cfg<8, 8, 2, 32, 2, 4, 4>;
using Cfg26 = Cfg<4, 16, 3, 16, 3, 4, 4>;
using Cfg27 = Cfg<4, 16, 2, 24, 3, 4, 4>;
using Cfg28 = Cfg<4, 16, 2, 24, 3, 4, 4, true>;
using Cfg29 = Cfg<4, 16, 2, 16, 4, 4, 4>;
using Cfg30 = Cfg<4, 16, 2, 16, 4, 4, 4, true>;
// Adjoint shapes (cs_query_grad; tile_config 1-4, 0 = 2): the adjoint keeps
// three gradient sums per primitive, so its tiles hold fewer primitives
//   1: 4 x 8, 3 stages x 8 chunks, 3 CTAs/SM
//   2: 4 x 8, 3 stages x 16 chunks, 3 CTAs/SM, row pairs interleaved
//   3: 4 x 8, 2 stages x 24 chunks, 3 CTAs/SM, row pairs interleaved
//   4: 8 x 8, 2 stages x 16 chunks, 2 CTAs/SM, row pairs interleaved
using CfgGrad1 = Cfg<4, 8, 3, 8, 3>;
using CfgGrad2 = Cfg<4, 8, 3, 16, 3, 2, 2>;
using CfgGrad3 = Cfg<4, 8, 2, 24, 3, 2, 2>;
using CfgGrad4 = Cfg<8, 8, 2, 16, 2, 2, 2>;
// the fused forward + adjoint launch of sphere cost queries (cs_query_fwd_grad):
// 4 x 8, 2 x 24, 3 CTAs/SM, row pairs, persistent (SMs x 3 CTAs take tiles
// from a counter)
using CfgGradF = Cfg<4, 8, 2, 24, 3, 2, 2, true>;
constexpr int kDefaultGradTile = 2;
static const int kTileIds[] = {1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30};
static_assert(sizeof(kTileIds) / sizeof(kTileIds[0]) <= 64, "callers hold up to 64 shape ids");
constexpr int kDefaultTile = 18;
constexpr int kSmallBatchTile = 23;
constexpr int kSmallBatchQ = 1 << 17;

int tile_configs(int32_t *ids, int32_t cap) {
    int n = (int)(sizeof(kTileIds) / sizeof(kTileIds[0]));
    for (int i = 0; i < n && i < cap; ++i) ids[i] = kTileIds[i];
    return n;
}

template <int PRIM, class C, int MODE, bool GRAD, bool EX = false, int SH = 0>
static cudaError_t launch_eval_t(const EvalArgs &a, cudaStream_t s) {
    constexpr int TQ = C::NCW * C::QW;
    const int ntiles = (a.Q + TQ - 1) / TQ;
    const size_t smem = sizeof(EvalSmem<C>);
    auto kern = k_eval<PRIM, C, MODE, GRAD, EX, SH>;
    EvalArgs b = a;
    b.ntiles = ntiles;
    int grid = ntiles;
    if constexpr (C::PERSIST) {
        // the tile counter is the word after the stream's error word; it
        // starts every launch at zero
        b.tile_ctr = reinterpret_cast<int *>(a.err + 1);
        cudaError_t e0 = cudaMemsetAsync(b.tile_ctr, 0, sizeof(int), s);
        if (e0 != cudaSuccess) return e0;
        grid = std::min(ntiles, std::max(a.num_sms, 1) * C::MINB);
    }
    // the shared-memory limit is a per-device attribute of the kernel: set it
    // once per (instantiation, device); bit d of `attr` records device d
    // (devices from 64 up set it on every launch, which is idempotent)
    static std::atomic<unsigned long long> attr{0ull};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(attr.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr.fetch_or(bit, std::memory_order_release);
    }
    kern<<<grid, (C::NCW + 1) * 32, smem, s>>>(b);
    count_launches(1);
    return cudaGetLastError();
}

template <int PRIM, class C>
static cudaError_t launch_mode(const EvalArgs &a, cudaStream_t s) {
    if (a.k.mode == CS_METRIC_FLAGS) {  // one small and one large shape serve the flags mode
        if (a.Q <= kSmallBatchQ) return launch_eval_t<PRIM, Cfg23, 3, false>(a, s);
        return launch_eval_t<PRIM, Cfg18, 3, false>(a, s);
    }
    const int mode = a.k.mode == CS_METRIC_MIN_S2 ? 1 : a.k.mode == CS_METRIC_SOFTMIN_S2 ? 2 : 0;
    if (mode == 0) return launch_eval_t<PRIM, C, 0, false>(a, s);
    if (mode == 1) return launch_eval_t<PRIM, C, 1, false>(a, s);
    return launch_eval_t<PRIM, C, 2, false>(a, s);
}

// A conservatism sweep's sphere cost launches on the shapes whose warps take
// consecutive row pairs (the n_sigma copies of a primitive) share the
// copies' geometry (over row quads where the layout keeps them together);
// sphere cost launches with k_thr = 0 keep a running minimum instead of the
// in-collision count; every other launch keeps the plain evaluation.
template <int PRIM, class C>
static cudaError_t launch_mode_sweep(const EvalArgs &a, cudaStream_t s) {
    if constexpr (PRIM == 0 && C::GROUP == 4 && C::IL == 4) {
        const bool cost = a.k.mode == CS_METRIC_MEAN_COST || a.k.mode == CS_METRIC_SUM_COST;
        if (a.k.sweep > 1 && a.k.sweep % 4 == 0 && cost)
            return a.k.k_thr == 0 ? launch_eval_t<PRIM, C, 0, false, false, kShGeom | kShK0 | kShQuad>(a, s)
                                  : launch_eval_t<PRIM, C, 0, false, false, kShGeom | kShQuad>(a, s);
    }
    if constexpr (PRIM == 0 && (C::GROUP == 2 || (C::GROUP == 4 && C::IL == 4)) && C::IL != 1) {
        const bool cost = a.k.mode == CS_METRIC_MEAN_COST || a.k.mode == CS_METRIC_SUM_COST;
        if (a.k.sweep > 1 && cost)
            return a.k.k_thr == 0 ? launch_eval_t<PRIM, C, 0, false, false, kShGeom | kShK0>(a, s)
                                  : launch_eval_t<PRIM, C, 0, false, false, kShGeom>(a, s);
    }
    if constexpr (PRIM == 0) {
        const bool cost = a.k.mode == CS_METRIC_MEAN_COST || a.k.mode == CS_METRIC_SUM_COST;
        if (cost && a.k.k_thr == 0) return launch_eval_t<PRIM, C, 0, false, false, kShK0>(a, s);
    }
    return launch_mode<PRIM, C>(a, s);
}

template <int PRIM, class C>
static cudaError_t launch_grad(const EvalArgs &a, int mode, cudaStream_t s) {
    if (mode == 0) return launch_eval_t<PRIM, C, 0, true>(a, s);
    if (mode == 1) return launch_eval_t<PRIM, C, 1, true>(a, s);
    return launch_eval_t<PRIM, C, 2, true>(a, s);
}

// An adjoint launch that also writes forward outputs (cs_query_fwd_grad).
static bool fused_forward(const EvalArgs &a) { return a.out_metric || a.out_collide || a.out_count; }

// The exact variance (cs_params.exact_variance) runs the default shapes only:
// shape 23 up to 2^17 rows, 18 above (flags mode likewise), adjoint shape 2.
template <int PRIM>
static cudaError_t launch_exact(const EvalArgs &a, bool grad, cudaStream_t s) {
    const int mode = a.k.mode == CS_METRIC_MIN_S2 ? 1 : a.k.mode == CS_METRIC_SOFTMIN_S2 ? 2 : 0;
    if constexpr (PRIM == 0) {
        if (grad && mode == 0 && fused_forward(a)) return launch_eval_t<PRIM, CfgGrad2, 0, true, true, kShFwd>(a, s);
    }
    if (grad) {
        if (mode == 0) return launch_eval_t<PRIM, CfgGrad2, 0, true, true>(a, s);
        if (mode == 1) return launch_eval_t<PRIM, CfgGrad2, 1, true, true>(a, s);
        return launch_eval_t<PRIM, CfgGrad2, 2, true, true>(a, s);
    }
    const bool small = a.Q <= kSmallBatchQ;
    if (a.k.mode == CS_METRIC_FLAGS)
        return small ? launch_eval_t<PRIM, Cfg23, 3, false, true>(a, s) : launch_eval_t<PRIM, Cfg18, 3, false, true>(a, s);
    if (mode == 0)
        return small ? launch_eval_t<PRIM, Cfg23, 0, false, true>(a, s) : launch_eval_t<PRIM, Cfg18, 0, false, true>(a, s);
    if (mode == 1)
        return small ? launch_eval_t<PRIM, Cfg23, 1, false, true>(a, s) : launch_eval_t<PRIM, Cfg18, 1, false, true>(a, s);
    return small ? launch_eval_t<PRIM, Cfg23, 2, false, true>(a, s) : launch_eval_t<PRIM, Cfg18, 2, false, true>(a, s);
}

template <int PRIM>
static cudaError_t launch_prim(const EvalArgs &a, bool grad, int tile, cudaStream_t s) {
    if (a.k.exact) return launch_exact<PRIM>(a, grad, s);
    if (grad) {
        const int mode = a.k.mode == CS_METRIC_MIN_S2 ? 1 : a.k.mode == CS_METRIC_SOFTMIN_S2 ? 2 : 0;
        if constexpr (PRIM == 0) {
            // forward outputs in the same launch: its own persistent shape
            if (mode == 0 && fused_forward(a)) return launch_eval_t<PRIM, CfgGradF, 0, true, false, kShFwd>(a, s);
        }
        const int gt = (tile >= 1 && tile <= 4) ? tile : kDefaultGradTile;
        if (gt == 1) return launch_grad<PRIM, CfgGrad1>(a, mode, s);
        if (gt == 3) return launch_grad<PRIM, CfgGrad3>(a, mode, s);
        if (gt == 4) return launch_grad<PRIM, CfgGrad4>(a, mode, s);
        return launch_grad<PRIM, CfgGrad2>(a, mode, s);
    }
    switch (tile) {
        case 2: return launch_mode<PRIM, Cfg2>(a, s);
        case 3: return launch_mode<PRIM, Cfg3>(a, s);
        case 4: return launch_mode<PRIM, Cfg4>(a, s);
        case 5: return launch_mode<PRIM, Cfg5>(a, s);
        case 6: return launch_mode<PRIM, Cfg6>(a, s);
        case 7: return launch_mode<PRIM, Cfg7>(a, s);
        case 8: return launch_mode<PRIM, Cfg8>(a, s);
        case 9: return launch_mode<PRIM, Cfg9>(a, s);
        case 10: return launch_mode<PRIM, Cfg10>(a, s);
        case 11: return launch_mode<PRIM, Cfg11>(a, s);
        case 12: return launch_mode<PRIM, Cfg12>(a, s);
        case 13: return launch_mode<PRIM, Cfg13>(a, s);
        case 14: return launch_mode<PRIM, Cfg14>(a, s);
        case 15: return launch_mode_sweep<PRIM, Cfg15>(a, s);
        case 16: return launch_mode<PRIM, Cfg16>(a, s);
        case 17: return launch_mode<PRIM, Cfg17>(a, s);
        case 18: return launch_mode_sweep<PRIM, Cfg18>(a, s);
        case 19: return launch_mode_sweep<PRIM, Cfg19>(a, s);
        case 20: return launch_mode<PRIM, Cfg20>(a, s);
        case 21: return launch_mode<PRIM, Cfg21>(a, s);
        case 22: return launch_mode_sweep<PRIM, Cfg22>(a, s);
        case 23: return launch_mode_sweep<PRIM, Cfg23>(a, s);
        case 24: return launch_mode_sweep<PRIM, Cfg24>(a, s);
        case 25: return launch_mode_sweep<PRIM, Cfg25>(a, s);
        case 26: return launch_mode_sweep<PRIM, Cfg26>(a, s);
        case 27: return launch_mode_sweep<PRIM, Cfg27>(a, s);
        case 28: return launch_mode_sweep<PRIM, Cfg28>(a, s);
        case 29: return launch_mode_sweep<PRIM, Cfg29>(a, s);
        case 30: return launch_mode_sweep<PRIM, Cfg30>(a, s);
        default: return launch_mode<PRIM, Cfg1>(a, s);
    }
}

cudaError_t launch_eval(int prim_type, const EvalArgs &a, bool grad, int tile_cfg, int num_sms,
                        cudaStream_t s) {
    (void)num_sms;
    // default forward shape: one primitive row of eight per tile for batches
    // up to 2^17 rows (more, tighter tiles: small or sparse batches fill the
    // GPU and stage less), shape 18 above
    const int tile = tile_cfg > 0 ? tile_cfg : grad ? 0 : (a.Q <= kSmallBatchQ ? kSmallBatchTile : kDefaultTile);
    return prim_type == CS_PRIM_SPHERE ? launch_prim<0>(a, grad, tile, s) : launch_prim<1>(a, grad, tile, s);
}

cudaError_t run_eval(int prim_type, const SceneDev &sc, const float4 *qrec, const float *qns,
                     const uint32_t *perm, int Q, const cs_params &p, float *out_metric,
                     uint8_t *out_collide, int32_t *out_count, const float *grad_out,
                     float *grad_centres, unsigned *err, int num_sms, long long polls,
                     cudaStream_t s, unsigned *gflags) {
    EvalArgs a;
    a.sc = sc;
    a.qrec = qrec;
    a.qns = qns;
    a.perm = perm;
    a.Q = Q;
    a.S = sweep_blocks(p);
    a.Qb = Q / a.S;
    for (int k = 0; k < 8; ++k) a.sw.v[k] = k < a.S ? p.sweep_nsigma[k] : 0.f;
    a.k = make_consts(p);
    a.out_metric = out_metric;
    a.out_collide = out_collide;
    a.out_count = out_count;
    a.grad_out = grad_out;
    a.grad_centres = grad_centres;
    a.err = err;
    a.stats = p.out_pair_stats;
    a.kstats = p.out_kernel_stats;
    a.wait_polls = polls;
    a.gflags = gflags;
    a.num_sms = num_sms;
    a.tile_ctr = nullptr;
    a.ntiles = 0;
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
        if (wait_phase(&bar, 0u, polls) < 0) atomicOr(err, kErrTimeout);
    }
}

cudaError_t run_wait_selftest(long long polls, unsigned *err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(polls, err);
    count_launches(1);
    return cudaGetLastError();
}

void launch_prep(const float *prims, int prim_type, int Q, const SceneDev &sc, float ns_scalar,
                 const float *ns_rows, Workspace &ws, uint32_t **perm_out, cudaStream_t s) {
    const int thr = 256, blk = (Q + thr - 1) / thr;
    uint32_t *perm;
    if (Q <= kBucketMaxQ) {
        // small batch: keys with the bucket histogram, scan, one scatter
        uint32_t *hist = ws.sort_hist;
        cudaMemsetAsync(hist, 0, 4 * ((size_t)kBuckets() + 1), s);
        k_prep_keys<<<blk, thr, 0, s>>>(prims, prim_type, Q, sc, ws.keys[0], ws.vals[0], hist);
        count_launches(1);
        scan_exclusive(hist, hist, (size_t)kBuckets() + 1, ws.scan_tmp, s);
        perm = ws.vals[1];
        k_bucket_scatter<<<blk, thr, 0, s>>>(ws.keys[0], Q, hist, perm);
        count_launches(1);
    } else {
        k_prep_keys<<<blk, thr, 0, s>>>(prims, prim_type, Q, sc, ws.keys[0], ws.vals[0], nullptr);
        count_launches(1);
        int res = radix_sort(ws.keys, ws.vals, (size_t)Q, 32, ws.sort_hist, ws.scan_tmp, s);
        perm = ws.vals[res];
    }
    k_prep_recs<<<blk, thr, 0, s>>>(prims, prim_type, Q, perm, ns_scalar, ns_rows, ws.qrec,
                                    ws.qns, ws.err);
    count_launches(1);
    *perm_out = perm;
}

void launch_group(const float *metric, const uint8_t *collide, int Q, int G, float *gm, uint8_t *gc,
                  cudaStream_t s, unsigned *err) {
    const int64_t ng = (Q + G - 1) / G;
    const int64_t threads = G >= kGroupWarpMin ? ng * 32 : ng;
    k_group<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(metric, collide, Q, G, gm, gc, err);
    count_launches(1);
}

}  // namespace cs
