// Exact-product sketches of the precision mode (RE_PREC_EXACT): the right sketch
// A*X (Algorithm 1 step 3) and the left sketch Y*(A X) (step 6) on the tcgen05
// tensor cores with every product exact and every sum exact, the only rounding
// being one at 2^-40 of the row's power-of-two scale.  This resolves sketched
// singular values far below the FP32 accumulation floor (about 3e-7 sigma_1),
// e.g. the eps = 1e-8 read-off on the ten-decade spectra of Sec. 6.
//
// One kernel computes D = P * Q^T over a contraction of length K, where
//   * P (M rows) is FP32 -- or an FP32 pair hi + lo for the left sketch, whose P
//     is A X -- and each row r has a power-of-two bound |p_rk| < 2^e_r;
//   * Q (N rows) is given as two BF16 digit slices: the embeddings' normals are
//     multiples of 2^-13 below 6 in magnitude (the generator's grid rounding),
//     so g = xi0 + xi1 with xi0 on the 2^-5 grid (|xi0| <= 6) and xi1 = g - xi0
//     on the 2^-13 grid (|xi1| <= 2^-6), both exact in BF16.
// The converter warps cut p' = p 2^-e_r (|p'| < 1) into five digits on the grids
// 2^-8, 2^-16, 2^-24, 2^-32, 2^-40 (delta_0 = n 2^-8 with |n| <= 256, the others
// |n| <= 129), each exact in BF16, by adding and subtracting 1.5 2^k (exact
// rounding to a grid); the part of p' below 2^-41 is dropped.  The products
// delta_s xi_t are then exact, and summed by level s + t into five TMEM
// accumulators:
//   L0 = sum delta_0 xi_0                    multiples of 2^-13
//   L1 = sum delta_0 xi_1 + delta_1 xi_0     multiples of 2^-21
//   L2 = sum delta_1 xi_1 + delta_2 xi_0     multiples of 2^-29
//   L3 = sum delta_2 xi_1 + delta_3 xi_0     multiples of 2^-37
//   L4 = sum delta_3 xi_1 + delta_4 xi_0     (rounded; below 2^-29 of L0)
// (the level-5 product delta_4 xi_1 is below 2^-46 and dropped).  One MMA per A
// digit slice s multiplies it with both Q slices at once (N = 2 NT, the two
// slices being adjacent rows of the Q stage), writing (s, 0) into L_s and (s, 1)
// into the next accumulator L_{s+1}: five MMAs per K step.  Each product of L0 ..
// L3 is at most 2^16 of its level's unit, so a partial sum stays an exactly
// representable FP32 integer multiple of the unit while it is below 2^24 units:
// the sums are exact, whatever order the tensor core adds them in.  Over a
// segment of 32768 terms the partial sums are random walks (the digits of the
// embedding are independent of P) with a standard deviation of at most 2^20.5
// units, so 2^24 is more than 11 standard deviations away.  L4 is rounded by FP32
// as it accumulates, far below 2^-40 of the result.
// After each segment the epilogue warps convert the accumulators to integers in
// units of 2^-40 (exact for L0..L3, L4 rounded), add them into the int64 output
// with atomic adds -- integer additions, so segments and tiles split between
// CTAs (stream-K) sum exactly and the result does not depend on the order -- and
// clear the accumulators for the next segment.  D_rq = T_rq 2^(e_r - 40);
// |T| < K 2^42.6 fits int64 for K <= 2^20.
//
// Warp roles (persistent, one CTA per SM, 128-row P tiles x NT (<= 64) Q rows,
// K chunks of 64, stream-K over (tile, chunk)):
//   warps 0-15  converters: warp (q, h, part) converts, for row 32q + lane, 16 K
//               (part) of half h (32 K) of every chunk into five digit slices in
//               TMEM (the MMA's A operand), two TMEM stages of 5 x 16 columns.
//   warps 16-19 epilogue: drains the accumulators into the int64 output.
//   warp 20     TMA producer of P (FP32 half chunks 128 x 32, 128B swizzle,
//               zero fill past the edges; the lo plane too in pair mode).
//   warp 21     TMA producer of the two Q digit slices (NT rows x 64 K each).
//   warp 22     TMEM allocation; one thread issues 5 tcgen05.mma (M = 128,
//               N = 2 NT or NT, K = 16, BF16 -> FP32) per K step.
// TMEM: accumulators L0..L4 at columns [0, 5 NT) (NT apart), A stages from 320.
// Every mbarrier wait is bounded in time (2 s): on expiry the kernel raises the
// error flag, every role drains what it has in flight and TMEM is freed.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kNTMax = 64;                 // Q rows per tile (MMA N)
constexpr int kConvParts = 2;                      // converter warps per (lane quarter, half chunk)
constexpr int kConvWarps = 8 * kConvParts;
constexpr int kEpiWarps = 4;
constexpr int kThreads = (kConvWarps + kEpiWarps + 3) * 32;
constexpr int kPProdWarp = kConvWarps + kEpiWarps;
constexpr int kQProdWarp = kPProdWarp + 1;
constexpr int kMmaWarp = kQProdWarp + 1;
constexpr uint32_t kHalfBytes = kBM * 32 * 4;     // 16 KB FP32 half chunk
constexpr int kRingMax = 8;                        // FP32 half-chunk ring: 8 slots (4 for pairs)
constexpr int kAStages = 2;                        // TMEM digit stages (one half chunk each)
constexpr int kQStages = 3;                        // Q chunk stages
constexpr int kLevels = 5;                         // accumulators L0..L4, NT columns each
constexpr uint32_t kAStageCol = kLevels * kNTMax;  // 320
constexpr uint32_t kAStageCols = 5 * 16;           // five slices x 32 K (16 columns of BF16 pairs)
constexpr uint32_t kTmemCols = 512;
constexpr int kSegChunks = 512;                    // 32768 K per exact segment
static_assert(kAStageCol + kAStages * kAStageCols <= kTmemCols, "TMEM budget");
static_assert(kNTMax * 2 <= 256, "MMA N");

struct ExParams {
    const int* rexp;          // e_r of every P row (|p_rk| < 2^e_r), -127 <= e_r <= 126
    int64_t M, K;
    int N;                    // valid Q rows of this launch (output columns)
    int NT;                   // MMA N (multiple of 16, <= 64)
    int ntn;                  // Q tiles
    int64_t tiles, kchunks;   // tiles = P tiles x Q tiles
    int q_row0;               // first Q row of this launch inside the slice array
    int q_slice_rows;         // rows per digit slice in the Q array
    unsigned long long* T;    // int64 output (M x ldt), added to atomically
    int64_t ldt;
    int* err;
};

__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }

// Round to the grid of spacing ulp(c) (c = 1.5 2^k), ties to even: exact when
// |x| < 2^(k-1).
__device__ __forceinline__ float grid(float x, float c) { return sub_rn(add_rn(x, c), c); }

// ---- digit extraction on packed FP32x2 values (each lane rounded exactly as the
// scalar add / subtract / multiply, no contraction)
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 grid2(f2 x, f2 c) { return sub2(add2(x, c), c); }

// The five digits delta_0..delta_4 of two values p' (|p'| < 1): d[s] holds digit s
// of both.  In pair mode p' = a + b (an FP32 pair, |b| <= ulp(a)/2): delta_0 and
// delta_1 come from a exactly, then b joins the residual (one rounding far below
// 2^-40).
template <bool kPair>
__device__ __forceinline__ void digits5x2(f2 a, f2 b, f2 (&d)[5]) {
    const f2 c8 = pk(49152.f, 49152.f), c16 = pk(192.f, 192.f), c24 = pk(0.75f, 0.75f),
             c32 = pk(0x1.8p-9f, 0x1.8p-9f), c40 = pk(0x1.8p-17f, 0x1.8p-17f);
    d[0] = grid2(a, c8);
    f2 r = sub2(a, d[0]);
    d[1] = grid2(r, c16);
    r = sub2(r, d[1]);
    if constexpr (kPair) r = add2(r, b);
    d[2] = grid2(r, c24);
    r = sub2(r, d[2]);
    d[3] = grid2(r, c32);
    r = sub2(r, d[3]);
    d[4] = grid2(r, c40);
}

// two packed pairs (k, k+1) and (k+2, k+3) of one digit -> two BF16x2 words
__device__ __forceinline__ void pack4(f2 p01, f2 p23, uint32_t& w0, uint32_t& w1) {
    float x0, x1, x2, x3;
    upk(p01, x0, x1);
    upk(p23, x2, x3);
    w0 = __byte_perm(__float_as_uint(x0), __float_as_uint(x1), 0x7632);
    w1 = __byte_perm(__float_as_uint(x2), __float_as_uint(x3), 0x7632);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }   // -126 <= e <= 127

template <bool kPair>
__global__ void __launch_bounds__(kThreads, 1) ex_sketch_kernel(const __grid_constant__ CUtensorMap pmap,
                                                                const __grid_constant__ CUtensorMap pmap_lo,
                                                                const __grid_constant__ CUtensorMap qmap,
                                                                const ExParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int kRing = kPair ? kRingMax / 2 : kRingMax;
    __shared__ __align__(8) uint64_t r_full[kRingMax], r_empty[kRingMax];
    __shared__ __align__(8) uint64_t a_full[kAStages], a_empty[kAStages];
    __shared__ __align__(8) uint64_t q_full[kQStages], q_empty[kQStages];
    __shared__ __align__(8) uint64_t accf, acce, done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NP = kPair ? 2 : 1;                          // FP32 planes
    const uint32_t q_slice_bytes = (uint32_t)p.NT * kBK * 2;   // one digit slice of a chunk
    const uint32_t q_stage = (2 * q_slice_bytes + 1023u) & ~1023u;
    unsigned char* ring = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* qbuf = ring + (size_t)kRing * NP * kHalfBytes;

    if (tid == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&r_full[i], 1);
            mbar_init(&r_empty[i], 4 * kConvParts * 32);
        }
        for (int i = 0; i < kAStages; ++i) {
            mbar_init(&a_full[i], 4 * kConvParts * 32);
            mbar_init(&a_empty[i], 1);
        }
        for (int i = 0; i < kQStages; ++i) {
            mbar_init(&q_full[i], 1);
            mbar_init(&q_empty[i], 1);
        }
        mbar_init(&accf, 1);
        mbar_init(&acce, kEpiWarps * 32);
        mbar_init(&done_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem;

    // stream-K: this CTA owns chunks [c_begin, c_end) of the tile-major (tile, chunk) order
    const int64_t K = p.kchunks;
    const int64_t c_total = p.tiles * K;
    const int64_t c_begin = (int64_t)blockIdx.x * c_total / gridDim.x;
    const int64_t c_end = ((int64_t)blockIdx.x + 1) * c_total / gridDim.x;
    const int64_t total_chunks = c_end - c_begin;
    const int64_t t_first = c_begin / K;
    const int64_t ntile_span = total_chunks > 0 ? (c_end - 1) / K - t_first + 1 : 0;

    if (warp < kConvWarps) {
        // ---------------- converters: rows 32q + lane, 32 / kConvParts K of half h of every chunk
        constexpr int KP = 2 / kConvParts;                     // 16-K parts per converter warp
        const int q = warp & 3, h = (warp >> 2) & 1, part0 = (warp >> 3) * KP;
        const int r = 32 * q + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        int64_t mt = t_first / p.ntn, kc = c_begin % K;      // stepped below, no division in the loop
        int nt = (int)(t_first % p.ntn);
        int64_t cur_mt = -1;
        float scale = 1.f;
        for (int64_t g = 0; g < total_chunks; ++g) {
            const int64_t hg = 2 * g + h;
            const int sa = (int)(hg % kAStages);
            const int rs = (int)(hg % kRing);
            bool ok = mbar_wait(&a_empty[sa], (uint32_t)((hg / kAStages) & 1) ^ 1u, &s_abort, p.err);
            if (ok) ok = mbar_wait(&r_full[rs], (uint32_t)((hg / kRing) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;
            if (mt != cur_mt) {
                cur_mt = mt;
                const int64_t row = mt * kBM + r;
                scale = row < p.M ? pow2f(-p.rexp[row]) : 0.f;
            }
            // row r of the 128B-swizzled half tile: 16-byte chunk c sits at slot c ^ (r & 7)
            const unsigned char* src = ring + (size_t)rs * NP * kHalfBytes + (size_t)r * 128;
            tc_fence_after();
#pragma unroll
            for (int pi = 0; pi < KP; ++pi) {                  // 16 K per part
                const int part = part0 + pi;
                uint32_t w[5][8];
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {
                    const int cc = 4 * part + c4;
                    const float4 v = *reinterpret_cast<const float4*>(src + ((cc ^ (r & 7)) << 4));
                    float4 vl = make_float4(0.f, 0.f, 0.f, 0.f);
                    if constexpr (kPair) vl = *reinterpret_cast<const float4*>(src + kHalfBytes + ((cc ^ (r & 7)) << 4));
                    const f2 sc = pk(scale, scale);
                    f2 d01[5], d23[5];
                    digits5x2<kPair>(mul2(pk(v.x, v.y), sc), mul2(pk(vl.x, vl.y), sc), d01);
                    digits5x2<kPair>(mul2(pk(v.z, v.w), sc), mul2(pk(vl.z, vl.w), sc), d23);
#pragma unroll
                    for (int s = 0; s < 5; ++s) pack4(d01[s], d23[s], w[s][2 * c4], w[s][2 * c4 + 1]);
                }
                if (pi == KP - 1) mbar_arrive(&r_empty[rs]);   // all parts read: the slot may refill
                // A operand in TMEM: lane = row, column = two consecutive k; slice s of
                // stage sa at kAStageCol + 80 sa + 16 s, this part at + 8 part
                const uint32_t col = kAStageCol + kAStageCols * (uint32_t)sa + 8u * (uint32_t)part;
#pragma unroll
                for (int s = 0; s < 5; ++s) tmem_st8(lane_base + col + 16u * (uint32_t)s, w[s]);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&a_full[sa]);
            if (++kc == K) {
                kc = 0;
                if (++nt == p.ntn) {
                    nt = 0;
                    ++mt;
                }
            }
        }
    } else if (warp == kPProdWarp) {
        // ---------------- TMA producer of P half chunks (both planes in pair mode)
        if (lane == 0) {
            int64_t issued = 0;
            int64_t mt = t_first / p.ntn, kc = c_begin % K;
            int nt = (int)(t_first % p.ntn);
            for (int64_t hg = 0; hg < 2 * total_chunks; ++hg) {
                const int rs = (int)(hg % kRing);
                if (!mbar_wait(&r_empty[rs], (uint32_t)((hg / kRing) & 1) ^ 1u, &s_abort, p.err)) break;
                // the converters read this slot through the generic proxy; order those
                // reads before the TMA (async proxy) overwrites it
                fence_proxy_async();
                unsigned char* dst = ring + (size_t)rs * NP * kHalfBytes;
                mbar_arrive_expect_tx(&r_full[rs], NP * kHalfBytes);
                tma_load_2d(dst, &pmap, (int)(kc * kBK + 32 * (hg & 1)), (int)(mt * kBM), &r_full[rs]);
                if constexpr (kPair)
                    tma_load_2d(dst + kHalfBytes, &pmap_lo, (int)(kc * kBK + 32 * (hg & 1)), (int)(mt * kBM),
                                &r_full[rs]);
                ++issued;
                if ((hg & 1) && ++kc == K) {
                    kc = 0;
                    if (++nt == p.ntn) {
                        nt = 0;
                        ++mt;
                    }
                }
            }
            for (int64_t hg = std::max<int64_t>(0, issued - kRing); hg < issued; ++hg)
                mbar_drain(&r_full[hg % kRing], (uint32_t)((hg / kRing) & 1));
        }
    } else if (warp == kQProdWarp) {
        // ---------------- TMA producer of the Q digit slices
        if (lane == 0) {
            int64_t issued = 0;
            int64_t kc = c_begin % K;
            int nt = (int)(t_first % p.ntn);
            for (int64_t g = 0; g < total_chunks; ++g) {
                const int sq = (int)(g % kQStages);
                if (!mbar_wait(&q_empty[sq], (uint32_t)((g / kQStages) & 1) ^ 1u, &s_abort, p.err)) break;
                unsigned char* dst = qbuf + (size_t)sq * q_stage;
                const int y0 = p.q_row0 + nt * p.NT;
                mbar_arrive_expect_tx(&q_full[sq], 2 * q_slice_bytes);
                tma_load_2d(dst, &qmap, (int)(kc * kBK), y0, &q_full[sq]);
                tma_load_2d(dst + q_slice_bytes, &qmap, (int)(kc * kBK), p.q_slice_rows + y0, &q_full[sq]);
                ++issued;
                if (++kc == K) {
                    kc = 0;
                    if (++nt == p.ntn) nt = 0;
                }
            }
            for (int64_t g = std::max<int64_t>(0, issued - kQStages); g < issued; ++g)
                mbar_drain(&q_full[g % kQStages], (uint32_t)((g / kQStages) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            // one MMA per A digit slice s against both Q slices at once (N = 2 NT: the
            // two slices are contiguous rows of the Q stage) writes the products
            // (s, 0) and (s, 1) into the adjacent accumulators L_s and L_{s+1}: level
            // s + t lands in L_{s+t}.  The last slice takes Q slice 0 only.  The
            // epilogue zeroes the accumulators before each segment, so every MMA adds.
            const uint32_t idesc2 = idesc_bf16(2 * p.NT), idesc1 = idesc_bf16(p.NT);
            const uint32_t lstride = (uint32_t)p.NT;
            int64_t g = 0;            // chunk counter within this CTA's range
            int64_t nseg = 0;         // drains so far
            bool ok = true;
            for (int64_t j = 0; j < ntile_span && ok; ++j) {
                const int64_t t0 = (t_first + j) * K;
                const int64_t k0 = std::max(c_begin, t0) - t0, k1 = std::min(c_end, t0 + K) - t0;
                for (int64_t sk = k0; sk < k1 && ok; sk += kSegChunks) {
                    const int64_t sk1 = std::min(k1, sk + kSegChunks);
                    // the accumulators are zero once the epilogue has drained (and cleared) them
                    if (!mbar_wait(&acce, (uint32_t)(nseg & 1), &s_abort, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int64_t kc = sk; kc < sk1; ++kc, ++g) {
                        const int sq = (int)(g % kQStages);
                        if (!mbar_wait(&q_full[sq], (uint32_t)((g / kQStages) & 1), &s_abort, p.err)) {
                            ok = false;
                            break;
                        }
                        const uint32_t qst = smem_u32(qbuf + (size_t)sq * q_stage);
                        for (int h = 0; h < 2 && ok; ++h) {
                            const int64_t hg = 2 * g + h;
                            const int sa = (int)(hg % kAStages);
                            if (!mbar_wait(&a_full[sa], (uint32_t)((hg / kAStages) & 1), &s_abort, p.err)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t ast = tmem_base + kAStageCol + kAStageCols * (uint32_t)sa;
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t b = sw128_desc(qst + 32u * (uint32_t)(2 * h + kk));
                                const uint32_t a0 = ast + 8u * kk;
#pragma unroll
                                for (int sl = 0; sl < 4; ++sl)
                                    mma_bf16_ts(tmem_base + lstride * sl, a0 + 16u * sl, b, idesc2, 1u);
                                mma_bf16_ts(tmem_base + lstride * 4, a0 + 64u, b, idesc1, 1u);
                            }
                            mma_commit(&a_empty[sa]);
                        }
                        if (ok) mma_commit(&q_empty[sq]);
                    }
                    if (ok) {
                        mma_commit(&accf);
                        ++nseg;
                    }
                }
            }
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    } else {
        // ---------------- epilogue: each segment's sums, as int64, added into the output
        const int q = warp - kConvWarps;          // lane quarter of this epilogue warp
        const int r = 32 * q + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        const uint32_t ncols = (uint32_t)(kLevels * p.NT);
        // clear the accumulators (this warp's lanes), then let the MMAs start
        auto clear = [&]() {
            const uint32_t z[16] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            for (uint32_t c = 0; c < ncols; c += 16) tmem_st16(lane_base + c, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&acce);
        };
        clear();
        int64_t nseg = 0;
        bool ok = true;
        const uint32_t ls = (uint32_t)p.NT;
        for (int64_t j = 0; j < ntile_span && ok; ++j) {
            const int64_t tile = t_first + j;
            const int64_t t0 = tile * K;
            const int64_t k0 = std::max(c_begin, t0) - t0, k1 = std::min(c_end, t0 + K) - t0;
            const int64_t row = (tile / p.ntn) * kBM + r;
            const int n0 = (int)(tile % p.ntn) * p.NT;
            const int nvalid = std::min(p.NT, p.N - n0);
            unsigned long long* out = p.T + row * p.ldt + n0;
            for (int64_t sk = k0; sk < k1; sk += kSegChunks) {
                ok = mbar_wait(&accf, (uint32_t)(nseg & 1), &s_abort, p.err);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < p.NT; c += 8) {
                    float v0[8], v1[8], v2[8], v3[8], v4[8];
                    tmem_ld8(lane_base + (uint32_t)c, v0);
                    tmem_ld8(lane_base + ls + (uint32_t)c, v1);
                    tmem_ld8(lane_base + 2 * ls + (uint32_t)c, v2);
                    tmem_ld8(lane_base + 3 * ls + (uint32_t)c, v3);
                    tmem_ld8(lane_base + 4 * ls + (uint32_t)c, v4);
                    if (row < p.M) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            // units of 2^-40: L0 (2^-13), L1 (2^-21), L2 (2^-29), L3 (2^-37)
                            // exact, L4 rounded
                            const long long t = (__float2ll_rn(v0[i] * 8192.f) << 27) +
                                                (__float2ll_rn(v1[i] * 2097152.f) << 19) +
                                                (__float2ll_rn(v2[i] * 536870912.f) << 11) +
                                                (__float2ll_rn(v3[i] * 137438953472.f) << 3) +
                                                __float2ll_rn(v4[i] * 1099511627776.f);
                            if (c + i < nvalid && t != 0) atomicAdd(out + c + i, (unsigned long long)t);
                        }
                    }
                }
                tc_fence_before();
                clear();
                ++nseg;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ---- helpers around the kernel ------------------------------------------------

// e[r] = the smallest e with |A[r][k]| < 2^e for all k < K (0 for a zero row),
// from the largest |entry| as a bit pattern; status[0] |= 1 when a row holds Inf
// or NaN, |= 2 when an entry is 2^126 or more (outside the converter's scaling).
// One warp per row.
__global__ void row_exponent_kernel(const float* __restrict__ A, int64_t ld, int64_t M, int64_t K,
                                    int* __restrict__ e, int* __restrict__ status) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    const float* a = A + row * ld;
    uint32_t mx = 0;
    if ((ld & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) {
        const int64_t K4 = K >> 2;
        const float4* a4 = reinterpret_cast<const float4*>(a);
        for (int64_t k = lane; k < K4; k += 32) {
            const float4 v = __ldcs(a4 + k);
            mx = max(mx, max(max(__float_as_uint(v.x) & 0x7FFFFFFFu, __float_as_uint(v.y) & 0x7FFFFFFFu),
                             max(__float_as_uint(v.z) & 0x7FFFFFFFu, __float_as_uint(v.w) & 0x7FFFFFFFu)));
        }
        for (int64_t k = 4 * K4 + lane; k < K; k += 32) mx = max(mx, __float_as_uint(a[k]) & 0x7FFFFFFFu);
    } else {
        for (int64_t k = lane; k < K; k += 32) mx = max(mx, __float_as_uint(a[k]) & 0x7FFFFFFFu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
        int ex = 0;
        if (mx >= 0x7F800000u) atomicOr(status, 1);
        else if (mx != 0u) ex = (int)(mx >> 23) - 126;     // |a| in [2^(E-127), 2^(E-126))
        if (ex > 126) {
            atomicOr(status, 2);
            ex = 126;
        }
        e[row] = ex < -126 ? -126 : ex;
    }
}

// The two digit slices of Gaussian normals, K-major: D[t][row][k] for rows
// [0, rows) of the slice array (slice stride slice_rows x ld), k < kpad (zero
// for k >= kvalid).  Entry (row, k) is the normal of the embedding with
// (long index, short index) = (k, row0 + row): X(k, j) for X^T (stream GX) or
// Y(q, i) with i = k for Y (stream GY).  xi0 = g on the 2^-5 grid, xi1 = g - xi0.
__global__ void normal_digits_kernel(uint64_t seed, uint32_t stream, int64_t kvalid, int64_t kpad, int row0,
                                     int rows, uint16_t* __restrict__ D, int64_t ld, int64_t slice_rows) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int g0 = row0 >> 2;
    const int ng = (row0 + rows + 3) / 4 - g0;
    if (idx >= kpad * ng) return;
    const int64_t k = idx % kpad;
    const int g = g0 + (int)(idx / kpad);
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (k < kvalid) normals4((uint32_t)k, (uint32_t)g, stream, seed, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int row = 4 * g + t - row0;
        if (row < 0 || row >= rows) continue;
        const float x0 = __fsub_rn(__fadd_rn(z[t], 0x1.8p18f), 0x1.8p18f);   // grid 2^-5
        const float x1 = __fsub_rn(z[t], x0);
        D[(int64_t)row * ld + k] = (uint16_t)(__float_as_uint(x0) >> 16);
        D[(slice_rows + row) * ld + k] = (uint16_t)(__float_as_uint(x1) >> 16);
    }
}

// T (int64, units of 2^-40 of 2^e_r, row-major M x ldt) -> FP32 pair planes of
// the transposed result (column c of the result = row c of the planes, ld ldp)
// and optionally FP64 values (row-major, ldv); cexp[c] = max over rows of the
// exponent e with |value| < 2^e (atomicMax; the planes feed the left sketch).
// 32 x 32 tiles through shared memory so both sides are coalesced.
__global__ void ex_finalize_kernel(const long long* __restrict__ T, int64_t ldt, const int* __restrict__ rexp,
                                   int64_t M, int N, float* __restrict__ Phi, float* __restrict__ Plo, int64_t ldp,
                                   double* __restrict__ V, int64_t ldv, int* __restrict__ cexp) {
    __shared__ float shi[32][33], slo[32][33];
    __shared__ int sexp[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;     // 32 x 8 threads
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    if (threadIdx.x < 32) sexp[threadIdx.x] = -1000;
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int c = c0 + tx;
        float hi = 0.f, lo = 0.f;
        if (r < M && c < N) {
            const double v = ldexp((double)T[r * ldt + c], rexp[r] - 40);
            hi = (float)v;
            lo = (float)(v - (double)hi);
            if (V) V[r * ldv + c] = v;
            const uint32_t b = __float_as_uint(hi) & 0x7FFFFFFFu;
            if (b != 0u) atomicMax(&sexp[tx], (int)(b >> 23) - 126);
        }
        shi[i][tx] = hi;
        slo[i][tx] = lo;
    }
    __syncthreads();
    if (threadIdx.x < 32 && c0 + (int)threadIdx.x < N && sexp[threadIdx.x] > -1000)
        atomicMax(&cexp[c0 + threadIdx.x], sexp[threadIdx.x]);
    if (!Phi) return;
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i;
        const int64_t r = r0 + tx;
        if (c < N && r < M) {
            Phi[(int64_t)c * ldp + r] = shi[tx][i];
            Plo[(int64_t)c * ldp + r] = slo[tx][i];
        }
    }
}

// The left sketch's T (rows = A X columns c, columns = Y rows q) -> core[q][c]
// (FP64 row-major), value T 2^(cexp[c] - 40).
__global__ void ex_core_finalize_kernel(const long long* __restrict__ T, int64_t ldt, const int* __restrict__ cexp,
                                        int C, int Q, int c_off, int q_off, double* __restrict__ core,
                                        int64_t ld_core) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)C * Q) return;
    const int q = (int)(idx / C), c = (int)(idx % C);
    core[(int64_t)(q_off + q) * ld_core + c_off + c] =
        ldexp((double)T[(int64_t)c * ldt + q], cexp[c_off + c] - 40);
}

// FP64 row-major values -> pair planes of the transpose and column exponents
// (the caller's earlier columns of A X when a sketch step appends).
__global__ void f64_pairs_kernel(const double* __restrict__ V, int64_t ldv, int64_t M, int N, float* __restrict__ Phi,
                                 float* __restrict__ Plo, int64_t ldp, int* __restrict__ cexp) {
    __shared__ float shi[32][33], slo[32][33];
    __shared__ int sexp[32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    if (threadIdx.x < 32) sexp[threadIdx.x] = -1000;
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int64_t r = r0 + i;
        const int c = c0 + tx;
        float hi = 0.f, lo = 0.f;
        if (r < M && c < N) {
            const double v = V[r * ldv + c];
            hi = (float)v;
            lo = (float)(v - (double)hi);
            const uint32_t b = __float_as_uint(hi) & 0x7FFFFFFFu;
            if (b != 0u) atomicMax(&sexp[tx], (int)(b >> 23) - 126);
        }
        shi[i][tx] = hi;
        slo[i][tx] = lo;
    }
    __syncthreads();
    if (threadIdx.x < 32 && c0 + (int)threadIdx.x < N && sexp[threadIdx.x] > -1000)
        atomicMax(&cexp[c0 + threadIdx.x], sexp[threadIdx.x]);
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i;
        const int64_t r = r0 + tx;
        if (c < N && r < M) {
            Phi[(int64_t)c * ldp + r] = shi[tx][i];
            Plo[(int64_t)c * ldp + r] = slo[tx][i];
        }
    }
}

// column exponents left at the sentinel (an all-zero column) become 0
__global__ void fix_exp_kernel(int* __restrict__ e, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && e[i] < -126) e[i] = 0;
}

int g_ex_sms = 0;

}  // namespace

// ---- host side -----------------------------------------------------------------

cudaError_t launch_row_exponent(const float* A, int64_t ld, int64_t M, int64_t K, int* e, int* status,
                                cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    const int warps = 8;
    row_exponent_kernel<<<(unsigned)((M + warps - 1) / warps), warps * 32, 0, st>>>(A, ld, M, K, e, status);
    return cudaGetLastError();
}

cudaError_t launch_normal_digits(uint64_t seed, uint32_t stream, int64_t kvalid, int64_t kpad, int row0, int rows,
                                 uint16_t* D, int64_t ld, int64_t slice_rows, cudaStream_t st) {
    if (rows <= 0 || kpad <= 0) return cudaSuccess;
    const int ng = (row0 + rows + 3) / 4 - (row0 >> 2);
    const int64_t total = kpad * ng;
    normal_digits_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(seed, stream, kvalid, kpad, row0, rows, D,
                                                                        ld, slice_rows);
    return cudaGetLastError();
}

int ex_tile_n(int n) { return n >= kNTMax ? kNTMax : std::max(16, (n + 15) / 16 * 16); }

cudaError_t launch_ex_sketch(const float* P, const float* P_lo, int64_t ldp, int64_t M, int64_t K, const int* rexp,
                             const uint16_t* Qd, int64_t ldq, int q_slice_rows, int q_row0, int N,
                             unsigned long long* T, int64_t ldt, int* err_flag, cudaStream_t st, int* launches) {
    if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
    if (K > ((int64_t)1 << 20)) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap pmap, pmap_lo, qmap;
    const cuuint64_t pdim[2] = {(cuuint64_t)K, (cuuint64_t)M};
    const cuuint64_t pstride[1] = {(cuuint64_t)ldp * 4};
    const cuuint32_t pbox[2] = {32u, (cuuint32_t)kBM};
    CUresult r = enc(&pmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(P), pdim, pstride, pbox, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    pmap_lo = pmap;
    if (P_lo) {
        r = enc(&pmap_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(P_lo), pdim, pstride, pbox, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    const int NT = ex_tile_n(N);
    const cuuint64_t qdim[2] = {(cuuint64_t)ldq, (cuuint64_t)(2 * (int64_t)q_slice_rows)};
    const cuuint64_t qstride[1] = {(cuuint64_t)ldq * 2};
    const cuuint32_t qbox[2] = {(cuuint32_t)kBK, (cuuint32_t)NT};
    r = enc(&qmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(Qd), qdim, qstride, qbox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    ExParams p;
    p.rexp = rexp;
    p.M = M;
    p.K = K;
    p.N = N;
    p.NT = NT;
    p.ntn = (N + NT - 1) / NT;
    p.kchunks = (K + kBK - 1) / kBK;
    p.tiles = (M + kBM - 1) / kBM * p.ntn;
    p.q_row0 = q_row0;
    p.q_slice_rows = q_slice_rows;
    p.T = T;
    p.ldt = ldt;
    p.err = err_flag;
    const int np = P_lo ? 2 : 1;
    const int ring = P_lo ? kRingMax / 2 : kRingMax;
    const uint32_t q_stage = ((uint32_t)2 * NT * kBK * 2 + 1023u) & ~1023u;
    const size_t smem = (size_t)ring * np * kHalfBytes + (size_t)kQStages * q_stage + 1024;
    if (!g_ex_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_ex_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t grid = std::min<int64_t>(p.tiles * p.kchunks, g_ex_sms);
    cudaError_t e;
    if (P_lo) {
        e = allow_dynamic_smem(reinterpret_cast<const void*>(ex_sketch_kernel<true>));
        if (e != cudaSuccess) return e;
        ex_sketch_kernel<true><<<(unsigned)grid, kThreads, smem, st>>>(pmap, pmap_lo, qmap, p);
    } else {
        e = allow_dynamic_smem(reinterpret_cast<const void*>(ex_sketch_kernel<false>));
        if (e != cudaSuccess) return e;
        ex_sketch_kernel<false><<<(unsigned)grid, kThreads, smem, st>>>(pmap, pmap_lo, qmap, p);
    }
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_ex_finalize(const long long* T, int64_t ldt, const int* rexp, int64_t M, int N, float* Phi,
                               float* Plo, int64_t ldp, double* V, int64_t ldv, int* cexp, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + 31) / 32), (unsigned)((N + 31) / 32));
    ex_finalize_kernel<<<grid, 256, 0, st>>>(T, ldt, rexp, M, N, Phi, Plo, ldp, V, ldv, cexp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && cexp) {
        fix_exp_kernel<<<(N + 255) / 256, 256, 0, st>>>(cexp, N);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_ex_core_finalize(const long long* T, int64_t ldt, const int* cexp, int C, int Q, int c_off,
                                    int q_off, double* core, int64_t ld_core, cudaStream_t st) {
    if (C <= 0 || Q <= 0) return cudaSuccess;
    const int64_t total = (int64_t)C * Q;
    ex_core_finalize_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(T, ldt, cexp, C, Q, c_off, q_off, core,
                                                                            ld_core);
    return cudaGetLastError();
}

cudaError_t launch_f64_to_pairs(const double* V, int64_t ldv, int64_t M, int N, float* Phi, float* Plo, int64_t ldp,
                                int* cexp, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((unsigned)((M + 31) / 32), (unsigned)((N + 31) / 32));
    f64_pairs_kernel<<<grid, 256, 0, st>>>(V, ldv, M, N, Phi, Plo, ldp, cexp);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        fix_exp_kernel<<<(N + 255) / 256, 256, 0, st>>>(cexp, N);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace re
