// Batched right sketch on the tensor cores: AX_b = A_b X_b for thousands of
// independent blocks (Algorithm 1 step 3 per block), BF16x3 exactly as the
// single-matrix kernel (A split into three BF16 terms in TMEM, X BF16-exact,
// FP32 accumulation).  Work items are the 128-row tiles of the active blocks;
// one persistent CTA per SM walks its items and K chunks in one pipeline.
//
// Blocks come with any row pitch (a kernel block of n columns has ld = n), which
// one tensor map cannot address (its row pitch must be a multiple of 16 bytes).
// Every fourth row can: rows c, c+4, c+8, ... sit 16 ld bytes apart, and all of
// them start at the same offset (0..3 floats) past a 16-byte boundary.  So a
// row-major block gets four tensor maps, one per row class c, each starting at the
// 16-byte boundary at or below row c, and a tile's 128 rows are held in class
// order (tile row 32c + t = block row 4t + c of the tile's 128), which the
// epilogue undoes:
//   warps 12-15  A producers: per half chunk (128 rows x 32 k), row-major
//             blocks: one thread issues the four classes' boxes of 36 floats x 32
//             rows (the 32 values of each row with up to 3 before them) by TMA,
//             zero fill past the block's columns and rows.  Blocks stored
//             transposed: asynchronous copies of 16, 8 or 4 bytes along rows into
//             a k-major tile (cp.async, mbarrier arrive.noinc), zero fill past the
//             edges.
//             For a matrix-free kernel block (no A, 3-D points) they instead
//             stage the tile's 128 row points and the half chunk's 32 column
//             points (negated, as three coordinate arrays; padding far away so
//             that entries past the block come out as 1/sqrt(inf) = 0) and
//             arrive on the stage's mbarrier directly.
//   warp 16   X^T producer: 16-byte copies of the BF16 X^T chunk (N rows x 64 k).
//   warps 0-7 converters, warp 17 MMA issuer, warps 8-11 epilogue: as in the
//             single-matrix kernel.  Converter warp (q, h) of a row-major block
//             reads row class q, whose offset is one value for the whole warp, so
//             it takes the row's 32 values at a fixed position of its 36.  For a matrix-free block a
//             converter thread computes its row's 32 entries 1 / |x_r - y_k| in
//             FP32 from the staged points (differences, squares and fused
//             multiply-adds two entries at a time in packed FP32x2, the hardware
//             reciprocal square root), so the block is never in HBM.
// Every mbarrier wait is bounded in time (on expiry: error flag, drain, free
// TMEM, return).
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

using namespace tc;

constexpr int kBM = 128;
constexpr int kBK = 64;
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kAProdWarps = 4;
constexpr int kAProdWarp = kConvWarps + kEpiWarps;             // 12..15
constexpr int kBProdWarp = kAProdWarp + kAProdWarps;           // 16
constexpr int kMmaWarp = kBProdWarp + 1;                       // 17
constexpr int kThreads = (kMmaWarp + 1) * 32;                  // 576
constexpr uint32_t kClassPitch = 144;                          // row-class box: 36 floats per row
constexpr uint32_t kClassBytes = 32 * kClassPitch;             // 32 rows of one class
constexpr uint32_t kHalfBytes = 4 * kClassBytes;               // 18 KB half-chunk stage (other layouts use 16 KB)
constexpr uint32_t kTClassPitch = 528;                         // transposed block: 132 floats per stored row
constexpr uint32_t kTClassBytes = 8 * kTClassPitch;            // 8 stored rows of one class
constexpr int kAStages = 8;
constexpr int kStages = 2;
constexpr uint32_t kAStageCol = 256;
constexpr uint32_t kTmemCols = 512;
// matrix-free stage layout: 128 row points (float4) then the negated column
// coordinates x[32], y[32], z[32]; padding points sit at +-kFar
constexpr uint32_t kColPts = 128 * 16;
constexpr float kFar = 1e30f;

__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ unsigned long long add_x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long mul_x2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long fma_x2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// entries 1/|x_r - y_k| for two columns: (nx, ny, nz) hold the negated column
// coordinates of both, (x0, x1, x2) the row point in both halves
__device__ __forceinline__ void kernel_pair(unsigned long long x0, unsigned long long x1, unsigned long long x2,
                                            unsigned long long nx, unsigned long long ny, unsigned long long nz,
                                            float& e0, float& e1) {
    const unsigned long long dx = add_x2(x0, nx), dy = add_x2(x1, ny), dz = add_x2(x2, nz);
    const unsigned long long d2 = fma_x2(dz, dz, fma_x2(dy, dy, mul_x2(dx, dx)));
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(d2));
    // the hardware reciprocal square root (relative error below 2^-22): d2 is a
    // positive normal number for distinct points, +inf for padding (entry 0) and
    // 0 only for coincident points (entry +inf, reported as non-finite)
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(e0) : "f"(a));
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(e1) : "f"(b));
}

__device__ __forceinline__ int find_block(const int64_t* prefix, int count, int64_t item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// W-byte asynchronous copy (W = 4, 8, 16) of which src_bytes come from global, the rest zero
template <int W>
__device__ __forceinline__ void cp_async_w(uint32_t dst, const void* src, uint32_t src_bytes) {
    if constexpr (W == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(W), "r"(src_bytes)
                     : "memory");
}

// Copy width for a block: the widest of 16, 8, 4 bytes that every row start allows.
__device__ __forceinline__ int copy_width(const float* A, int64_t ld) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(A);
    if ((a & 15) == 0 && (ld & 3) == 0) return 16;
    if ((a & 7) == 0 && (ld & 1) == 0) return 8;
    return 4;
}

// One half chunk (rows row0.., k0..k0+31) of a row-major block into the 128B-swizzled
// layout (row r at r*128, 16-byte chunk c at c ^ (r & 7)); this warp copies rows
// rbase .. rbase+31; lanes cover (row, W-byte segment) pairs.  Rows past the block
// are zero-filled in a second loop, so the main loop has no row test.
// The block's pointer and sizes arrive by value: the copies' "memory" clobbers
// would otherwise make every loop iteration reload them from the descriptor.
struct BlockRef {
    const float* A;
    int64_t ld, rows, cols;
};

template <int W>
__device__ __forceinline__ void load_rows(const BlockRef D, int64_t row0, int64_t k0, int rbase, uint32_t dst0) {
    constexpr int SEG = 128 / W;                  // segments per 128-byte row
    constexpr int RPI = 32 / SEG;                 // rows per warp instruction
    const int lane = threadIdx.x & 31;
    const int seg = lane % SEG;
    const int64_t k = k0 + seg * (W / 4);
    const int64_t kleft = D.cols - k;             // columns left from k
    const uint32_t nb = kleft >= W / 4 ? (uint32_t)W : (kleft > 0 ? (uint32_t)kleft * 4u : 0u);
    const uint32_t byte = (uint32_t)seg * W;      // byte offset inside the 128-byte row
    const int nvalid = (int)std::max<int64_t>(0, std::min<int64_t>(32, D.rows - (row0 + rbase)));
    int i = lane / SEG;
    const float* src = D.A + (row0 + rbase + i) * D.ld + (nb ? k : 0);
    const int64_t step = (int64_t)RPI * D.ld;
#pragma unroll 4
    for (; i < nvalid; i += RPI, src += step) {
        const int rr = rbase + i;
        const uint32_t dst = dst0 + (uint32_t)rr * 128u + (((byte >> 4) ^ (uint32_t)(rr & 7)) << 4) + (byte & 15u);
        cp_async_w<W>(dst, nb ? src : D.A, nb);
    }
    for (; i < 32; i += RPI) {
        const int rr = rbase + i;
        const uint32_t dst = dst0 + (uint32_t)rr * 128u + (((byte >> 4) ^ (uint32_t)(rr & 7)) << 4) + (byte & 15u);
        cp_async_w<W>(dst, D.A, 0u);
    }
}

// One half chunk of a block stored transposed (oriented (row, k) = A[k * ld + row])
// into a k-major tile: k row kk at kk*512, 128 oriented rows contiguous; this warp
// copies k rows kbase .. kbase+7, lanes over W-byte segments of each.
template <int W>
__device__ __forceinline__ void load_cols(const BlockRef D, int64_t row0, int64_t k0, int kbase, uint32_t dst0) {
    constexpr int SEG = 512 / W;                  // segments per 512-byte k row
    constexpr int PER = W / 4;                    // floats per segment
    const int lane = threadIdx.x & 31;
    const int64_t rleft0 = D.rows - row0;         // oriented rows left from row0
    for (int kk = kbase; kk < kbase + 8; ++kk) {
        const int64_t k = k0 + kk;
        const bool kin = k < D.cols;
        const float* rowp = D.A + (kin ? k : 0) * D.ld + row0;
        const uint32_t dk = dst0 + (uint32_t)kk * 512u;
#pragma unroll
        for (int sg = lane; sg < SEG; sg += 32) {
            const int64_t rl = rleft0 - (int64_t)sg * PER;
            const uint32_t nb = !kin ? 0u : (rl >= PER ? (uint32_t)W : (rl > 0 ? (uint32_t)rl * 4u : 0u));
            cp_async_w<W>(dk + (uint32_t)sg * W, nb ? rowp + sg * PER : D.A, nb);
        }
    }
}

// the mbarrier receives one arrival when all prior cp.async of this thread land
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct TcBatchParams {
    const CUtensorMap* tmaps; // four row-class maps per block (row-major blocks with d[b].tmaps)
    const BatchDesc* d;
    int count;
    const int64_t* pre;       // prefix of the active blocks' 128-row tiles (count + 1 entries)
    const int* tb;            // block of each of those tiles (launch_compact_tiles)
    const uint16_t* xt;       // X^T pool
    int N;                    // MMA N (rows of each block's X^T)
    int S;                    // valid output columns
    float* ax;
    int64_t ldax;
    int col0;
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1) right_tc_batched_kernel(const TcBatchParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[kAStages], a_empty[kAStages];
    __shared__ __align__(8) uint64_t full_a[kStages], full_b[kStages], empty[kStages];
    __shared__ __align__(8) uint64_t accf[2], acce[2], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t items = p.pre[p.count];      // tiles of the active blocks (set on the device)
    const uint32_t b_stage = ((uint32_t)p.N * 128u + 1023u) & ~1023u;
    unsigned char* abuf = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* bbuf = abuf + (size_t)kAStages * kHalfBytes;

    if (tid == 0) {
        for (int i = 0; i < kAStages; ++i) {
            mbar_init(&a_full[i], kAProdWarps * 32);
            mbar_init(&a_empty[i], (kConvWarps / 2) * 32);   // the 4 converter warps of that half
        }
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full_a[i], kConvWarps * 32);
            mbar_init(&full_b[i], 32);
            mbar_init(&empty[i], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&accf[a], 1);
            mbar_init(&acce[a], kEpiWarps * 32);
        }
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

    if (warp < kConvWarps) {
        // ---------------- converters (as in the single-matrix kernel)
        const int q = warp & 3, h = warp >> 2;
        const int r = 32 * q + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        int64_t g = 0;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const int b = p.tb[it];
            const int64_t kch = p.d[b].kpad / kBK;
            const bool trans = p.d[b].trans != 0;
            const bool mfree = p.d[b].A == nullptr;
            const bool cls = p.d[b].tmaps == 1, tcls = p.d[b].tmaps == 2;
            // row class q's offset past its 16-byte boundary (one value for the warp)
            const int off = cls ? (int)((reinterpret_cast<uintptr_t>(p.d[b].A + (int64_t)q * p.d[b].ld) & 15u) >> 2) : 0;
            // stored transposed: each class's first value of this thread's oriented row r
            // (class c, stored row 4t + c at c * kTClassBytes + t * kTClassPitch)
            uint32_t tbase[4] = {0u, 0u, 0u, 0u};
            if (tcls) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t o = (uint32_t)((reinterpret_cast<uintptr_t>(p.d[b].A + (int64_t)c * p.d[b].ld) & 15u) >> 2);
                    tbase[c] = (uint32_t)c * kTClassBytes + 4u * (o + (uint32_t)r);
                }
            }
            for (int64_t kc = 0; kc < kch; ++kc, ++g) {
                const int s = (int)(g % kStages);
                ok = mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err);
                const int64_t hg = 2 * g + h;
                const int as = (int)(hg % kAStages);
                if (ok) ok = mbar_wait(&a_full[as], (uint32_t)((hg / kAStages) & 1), &s_abort, p.err);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const unsigned char* tile = abuf + (size_t)as * kHalfBytes;
                const uint32_t col = kAStageCol + 96u * (uint32_t)s + 16u * (uint32_t)h;
                if (mfree) {
                    // entries computed and stored to TMEM eight words (16 entries) at a time
                    const float4 xr = reinterpret_cast<const float4*>(tile)[r];
                    const unsigned long long x0 = pk(xr.x, xr.x), x1 = pk(xr.y, xr.y), x2 = pk(xr.z, xr.z);
                    const float* cx = reinterpret_cast<const float*>(tile + kColPts);
                    tc_fence_after();
#pragma unroll
                    for (int half = 0; half < 2; ++half) {
                        uint32_t h8[8], m8[8], l8[8];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const int cc = 4 * half + c;
                            const float4 gx = *reinterpret_cast<const float4*>(cx + 4 * cc);
                            const float4 gy = *reinterpret_cast<const float4*>(cx + 32 + 4 * cc);
                            const float4 gz = *reinterpret_cast<const float4*>(cx + 64 + 4 * cc);
                            float e0, e1, e2, e3;
                            kernel_pair(x0, x1, x2, pk(gx.x, gx.y), pk(gy.x, gy.y), pk(gz.x, gz.y), e0, e1);
                            kernel_pair(x0, x1, x2, pk(gx.z, gx.w), pk(gy.z, gy.w), pk(gz.z, gz.w), e2, e3);
                            split3(e0, e1, h8[2 * c], m8[2 * c], l8[2 * c]);
                            split3(e2, e3, h8[2 * c + 1], m8[2 * c + 1], l8[2 * c + 1]);
                        }
                        tmem_st8(lane_base + col + 8u * half, h8);
                        tmem_st8(lane_base + col + 32u + 8u * half, m8);
                        tmem_st8(lane_base + col + 64u + 8u * half, l8);
                    }
                    mbar_arrive(&a_empty[as]);
                } else {
                    float4 v[8];
                    if (cls) {
                        // class q, row lane: 36 floats at pitch 144 (granules 9 lane + c: eight
                        // consecutive lanes hit distinct bank groups); the row's values start at off
                        const float4* src = reinterpret_cast<const float4*>(tile + (size_t)q * kClassBytes +
                                                                            (size_t)lane * kClassPitch);
                        float4 w4[9];
#pragma unroll
                        for (int c = 0; c < 9; ++c) w4[c] = src[c];
                        if (off == 0) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[c] = w4[c];
                        } else if (off == 1) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[c] = make_float4(w4[c].y, w4[c].z, w4[c].w, w4[c + 1].x);
                        } else if (off == 2) {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[c] = make_float4(w4[c].z, w4[c].w, w4[c + 1].x, w4[c + 1].y);
                        } else {
#pragma unroll
                            for (int c = 0; c < 8; ++c) v[c] = make_float4(w4[c].w, w4[c + 1].x, w4[c + 1].y, w4[c + 1].z);
                        }
                    } else if (tcls) {
                        // k-major rows by class: value (kk, r) at tbase[kk % 4] + (kk / 4) * pitch;
                        // consecutive lanes read consecutive words
#pragma unroll
                        for (int c = 0; c < 8; ++c) {
                            const unsigned char* t = tile + (size_t)c * kTClassPitch;
                            v[c] = make_float4(*reinterpret_cast<const float*>(t + tbase[0]),
                                               *reinterpret_cast<const float*>(t + tbase[1]),
                                               *reinterpret_cast<const float*>(t + tbase[2]),
                                               *reinterpret_cast<const float*>(t + tbase[3]));
                        }
                    } else if (!trans) {
                        const unsigned char* src = tile + (size_t)r * 128;
#pragma unroll
                        for (int c = 0; c < 8; ++c) v[c] = *reinterpret_cast<const float4*>(src + ((c ^ (r & 7)) << 4));
                    } else {
                        // k-major tile: column r (consecutive lanes read consecutive words)
                        const float* src = reinterpret_cast<const float*>(tile) + r;
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            v[c] = make_float4(src[(4 * c) * 128], src[(4 * c + 1) * 128], src[(4 * c + 2) * 128],
                                               src[(4 * c + 3) * 128]);
                    }
                    mbar_arrive(&a_empty[as]);
                    uint32_t hi[16], mid[16], lo[16];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        split3(v[c].x, v[c].y, hi[2 * c], mid[2 * c], lo[2 * c]);
                        split3(v[c].z, v[c].w, hi[2 * c + 1], mid[2 * c + 1], lo[2 * c + 1]);
                    }
                    tc_fence_after();
                    tmem_st16(lane_base + col, hi);
                    tmem_st16(lane_base + col + 32u, mid);
                    tmem_st16(lane_base + col + 64u, lo);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&full_a[s]);
            }
        }
    } else if (warp >= kAProdWarp && warp < kAProdWarp + kAProdWarps) {
        // ---------------- A producers: W-byte cp.async (W from the block's alignment)
        const int pw = warp - kAProdWarp;
        int64_t hg = 0;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const int b = p.tb[it];
            const BatchDesc& D = p.d[b];
            const BlockRef B{D.A, D.ld, D.rows, D.cols};   // in registers for the whole tile
            const bool tr = D.trans != 0;
            const int64_t row0 = (it - p.pre[b]) * kBM;
            const int64_t kch = D.kpad / kBK;
            const bool mfree = B.A == nullptr;
            const int w = mfree ? 4 : copy_width(B.A, B.ld);
            // matrix-free: this thread's row point (row t = 32 pw + lane of the tile) is the
            // same for every K chunk, so it is loaded once per tile
            float4 rp = make_float4(kFar, kFar, kFar, 0.f);
            if (mfree && row0 + 32 * pw + lane < B.rows) {
                const float* xp = D.px + 3 * (row0 + 32 * pw + lane);
                rp = make_float4(xp[0], xp[1], xp[2], 0.f);
            }
            for (int64_t kc = 0; kc < kch && ok; ++kc) {
                for (int h = 0; h < 2; ++h, ++hg) {
                    const int as = (int)(hg % kAStages);
                    // matrix-free: the half chunk's column point (k0 + lane, negated) is
                    // loaded before the wait for the stage, so the load overlaps the wait
                    float nx = kFar, ny = kFar, nz = kFar;
                    if (mfree && pw == 0) {
                        const int64_t k = kc * kBK + 32 * h + lane;
                        if (k < B.cols) {
                            const float* yp = D.py + 3 * k;
                            nx = -yp[0];
                            ny = -yp[1];
                            nz = -yp[2];
                        }
                    }
                    ok = mbar_wait(&a_empty[as], (uint32_t)((hg / kAStages) & 1) ^ 1u, &s_abort, p.err);
                    if (!__all_sync(0xffffffffu, ok)) {
                        ok = false;
                        break;
                    }
                    const uint32_t dst0 = smem_u32(abuf + (size_t)as * kHalfBytes);
                    const int64_t k0 = kc * kBK + 32 * h;
                    if (D.tmaps) {
                        // the four row classes' boxes by TMA (one thread; the others arrive).
                        // Row-major: class c's 32 rows of the tile (x = k0, y = row0 / 4).
                        // Stored transposed: class c's 8 stored rows of the half chunk
                        // (x = row0, the tile's first oriented row; y = k0 / 4)
                        if (pw == 0 && lane == 0) {
                            // the converters read this stage through the generic proxy; order
                            // those reads before the TMA (async proxy) overwrites it
                            fence_proxy_async();
                            const bool rm = D.tmaps == 1;
                            const int64_t srows = rm ? B.rows : B.cols;     // stored rows
                            const uint32_t cb = rm ? kClassBytes : kTClassBytes;
                            int ncls = 0;
                            for (int c = 0; c < 4; ++c) ncls += srows > c ? 1 : 0;
                            mbar_arrive_expect_tx(&a_full[as], (uint32_t)ncls * cb);
                            for (int c = 0; c < 4; ++c)
                                if (srows > c)
                                    tma_load_2d(abuf + (size_t)as * kHalfBytes + (size_t)c * cb,
                                                p.tmaps + 4 * (int64_t)b + c, rm ? (int)k0 : (int)row0,
                                                rm ? (int)(row0 / 4) : (int)(k0 / 4), &a_full[as]);
                        } else {
                            mbar_arrive(&a_full[as]);
                        }
                        continue;
                    }
                    if (mfree) {
                        unsigned char* stg = abuf + (size_t)as * kHalfBytes;
                        reinterpret_cast<float4*>(stg)[32 * pw + lane] = rp;   // row point t of the tile
                        if (pw == 0) {                          // column point k0 + lane, negated
                            float* cs = reinterpret_cast<float*>(stg + kColPts);
                            cs[lane] = nx;
                            cs[32 + lane] = ny;
                            cs[64 + lane] = nz;
                        }
                        mbar_arrive(&a_full[as]);             // release: the staged points before the arrival
                        continue;
                    }
                    if (!tr) {
                        if (w == 16) load_rows<16>(B, row0, k0, 32 * pw, dst0);
                        else if (w == 8) load_rows<8>(B, row0, k0, 32 * pw, dst0);
                        else load_rows<4>(B, row0, k0, 32 * pw, dst0);
                    } else {
                        if (w == 16) load_cols<16>(B, row0, k0, 8 * pw, dst0);
                        else if (w == 8) load_cols<8>(B, row0, k0, 8 * pw, dst0);
                        else load_cols<4>(B, row0, k0, 8 * pw, dst0);
                    }
                    cp_async_arrive(&a_full[as]);
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok) {
            // aborted: let TMA loads already issued into this CTA's shared memory land
            const unsigned long long t0 = now_ns();
            while (now_ns() - t0 < 100000ull) {
            }
        }
    } else if (warp == kBProdWarp) {
        // ---------------- X^T producer: 16-byte cp.async, N rows x 128 bytes per chunk
        int64_t g = 0;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
            const int b = p.tb[it];
            const BatchDesc& D = p.d[b];
            const uint16_t* xt = p.xt + D.xt_off;
            const int64_t kch = D.kpad / kBK;
            for (int64_t kc = 0; kc < kch; ++kc, ++g) {
                const int s = (int)(g % kStages);
                ok = mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err);
                if (!__all_sync(0xffffffffu, ok)) {
                    ok = false;
                    break;
                }
                const uint32_t dst0 = smem_u32(bbuf + (size_t)s * b_stage);
                for (int t = lane; t < p.N * 8; t += 32) {
                    const int row = t >> 3, c = t & 7;
                    cp_async16(dst0 + (uint32_t)row * 128u + ((uint32_t)(c ^ (row & 7)) << 4),
                               xt + (int64_t)row * D.kpad + kc * kBK + 8 * c);
                }
                cp_async_arrive(&full_b[s]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(p.N);
            int64_t g = 0, j = 0;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
                const int b = p.tb[it];
                const int64_t kch = p.d[b].kpad / kBK;
                const int a = (int)(j & 1);
                if (!mbar_wait(&acce[a], (uint32_t)(((j >> 1) & 1) ^ 1), &s_abort, p.err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * p.N);
                for (int64_t kc = 0; kc < kch; ++kc, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!mbar_wait(&full_a[s], ph, &s_abort, p.err) || !mbar_wait(&full_b[s], ph, &s_abort, p.err)) {
                        ok = false;
                        break;
                    }
                    // X^T arrived through the generic proxy (cp.async): order it before the MMA's reads
                    fence_proxy_async();
                    tc_fence_after();
                    const uint32_t bst = smem_u32(bbuf + (size_t)s * b_stage);
                    const uint32_t ast = tmem_base + kAStageCol + 96u * (uint32_t)s;
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t bdesc = sw128_desc(bst + 32u * kk);
#pragma unroll
                        for (int term = 0; term < 3; ++term)
                            mma_bf16_ts(d_tmem, ast + 32u * term + 8u * kk, bdesc, idesc, (kc | kk | term) ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&accf[a]);
                ++j;
            }
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    } else {
        // ---------------- epilogue warps 8..11: TMEM lanes 32*(warp%4) ..
        const int q = warp & 3;
        int64_t j = 0;
        for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
            const int b = p.tb[it];
            const int a = (int)(j & 1);
            const bool ok = mbar_wait(&accf[a], (uint32_t)((j >> 1) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;   // tcgen05.ld is warp-wide
            tc_fence_after();
            const BatchDesc& D = p.d[b];
            // tile rows in class order for blocks fetched by row class (tile row 32q + lane
            // is block row 4 lane + q of the tile)
            const int64_t row = (it - p.pre[b]) * kBM + (D.tmaps == 1 ? 4 * lane + q : q * 32 + lane);
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * p.N);
            for (int c = 0; c < p.N; c += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c, v);
                if (row < D.rows) {
                    float* dst = p.ax + D.ax_off + row * p.ldax + p.col0 + c;
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        if (c + i < p.S) *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[a]);
            ++j;
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

// X_b^T[j][k] = bf16 normal X_b(k, col0 + j) for j < s, k < cols; zero elsewhere
// in the nxt x kpad region (one thread per (block-relative k, group of 4 columns)).
__global__ void gauss_xt_batched_kernel(const BatchDesc* __restrict__ d, int count, const int* __restrict__ active,
                                        int col0, int s, int nxt, uint16_t* __restrict__ pool) {
    const int b = blockIdx.y;
    if (b >= count || !active[b]) return;
    const BatchDesc D = d[b];
    uint16_t* xt = pool + D.xt_off;
    const int ng = nxt / 4;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < D.kpad * ng;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = idx % D.kpad;
        const int g = (int)(idx / D.kpad);
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (k < D.cols && 4 * g < s) normals4((uint32_t)k, (uint32_t)((col0 >> 2) + g), kStreamGX, D.seed, z);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * g + e;
            xt[(int64_t)j * D.kpad + k] = j < s ? (uint16_t)(__float_as_uint(z[e]) >> 16) : (uint16_t)0;
        }
    }
}

// act_pre[b] = number of 128-row tiles of the active blocks before b (one CTA).
__global__ void __launch_bounds__(1024) compact_tiles_kernel(const BatchDesc* __restrict__ d, int count,
                                                             const int* __restrict__ active,
                                                             int64_t* __restrict__ act_pre) {
    __shared__ int64_t s_part[1024];
    const int t = threadIdx.x;
    const int per = (count + 1023) / 1024;
    const int b0 = t * per, b1 = min(count, b0 + per);
    int64_t sum = 0;
    for (int b = b0; b < b1; ++b)
        if (active[b]) sum += (d[b].rows + kBM - 1) / kBM;
    s_part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {          // inclusive scan of the per-thread sums
        const int64_t v = t >= o ? s_part[t - o] : 0;
        __syncthreads();
        s_part[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? s_part[t - 1] : 0;
    for (int b = b0; b < b1; ++b) {
        act_pre[b] = run;
        if (active[b]) run += (d[b].rows + kBM - 1) / kBM;
    }
    if (t == 1023) act_pre[count] = s_part[1023];
}

// tile_block[t] = the active block holding tile t (t < act_pre[count]): one search
// per tile here instead of one per tile in every role of the sketch kernel
__global__ void tile_block_kernel(const int64_t* __restrict__ act_pre, int count, int64_t max_items,
                                  int* __restrict__ tile_block) {
    const int64_t items = min(act_pre[count], max_items);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < items; t += (int64_t)gridDim.x * blockDim.x)
        tile_block[t] = find_block(act_pre, count, t);
}

int g_bsms = 0;

}  // namespace

cudaError_t launch_compact_tiles(const BatchDesc* d, int count, const int* active, int64_t* act_pre,
                                 int* tile_block, int64_t max_items, cudaStream_t st) {
    if (count <= 0 || max_items <= 0) return cudaSuccess;
    compact_tiles_kernel<<<1, 1024, 0, st>>>(d, count, active, act_pre);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((max_items + 255) / 256, 1024);
    tile_block_kernel<<<(unsigned)blocks, 256, 0, st>>>(act_pre, count, max_items, tile_block);
    return cudaGetLastError();
}

cudaError_t launch_gauss_xt_batched(const BatchDesc* d, int count, const int* active, int col0, int s, int nxt,
                                    uint16_t* XTpool, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (s % 4 != 0 || col0 % 4 != 0 || nxt % 4 != 0 || count > 65535) return cudaErrorInvalidValue;
    gauss_xt_batched_kernel<<<dim3(8, (unsigned)count), 256, 0, st>>>(d, count, active, col0, s, nxt, XTpool);
    return cudaGetLastError();
}

size_t row_class_map_bytes() { return sizeof(CUtensorMap); }

bool encode_row_class_maps(const float* A, int64_t ld, int64_t rows, int64_t cols, int box_x, int box_y,
                           void* out) {
    EncodeTiled enc = encode_fn();
    if (!enc || !A || rows <= 0 || cols <= 0 || ld < cols) return false;
    CUtensorMap* maps = static_cast<CUtensorMap*>(out);
    for (int c = 0; c < 4; ++c) {
        std::memset(&maps[c], 0, sizeof(CUtensorMap));
        if (rows <= c) continue;                      // an empty class is never loaded
        const uintptr_t first = reinterpret_cast<uintptr_t>(A + (int64_t)c * ld);
        const uintptr_t base = first & ~(uintptr_t)15;
        const uint64_t off = (first - base) / 4;      // floats before row c's first value
        const cuuint64_t dim[2] = {(cuuint64_t)(off + cols), (cuuint64_t)((rows - c + 3) / 4)};
        const cuuint64_t stride[1] = {(cuuint64_t)ld * 16};
        const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = enc(&maps[c], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, reinterpret_cast<void*>(base), dim, stride,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

cudaError_t launch_right_tc_batched(const BatchDesc* d, int count, const int64_t* act_prefix, const int* tile_block,
                                    int64_t max_items, const uint16_t* XTpool, int s, float* AXpool, int64_t ldax,
                                    int col0, int* err_flag, const void* tmaps, cudaStream_t st) {
    if (max_items <= 0 || s <= 0 || count <= 0) return cudaSuccess;
    if (s > 256 || s % 8 != 0 || col0 % 4 != 0 || ldax % 4 != 0 || !err_flag || !tile_block)
        return cudaErrorInvalidValue;
    TcBatchParams p;
    p.tmaps = static_cast<const CUtensorMap*>(tmaps);
    p.d = d;
    p.count = count;
    p.pre = act_prefix;
    p.tb = tile_block;
    p.xt = XTpool;
    p.N = tc_mma_n(s);
    p.S = s;
    p.ax = AXpool;
    p.ldax = ldax;
    p.col0 = col0;
    p.err = err_flag;
    const size_t smem = (size_t)kHalfBytes * kAStages + (((size_t)p.N * 128 + 1023) & ~(size_t)1023) * kStages + 1024;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(right_tc_batched_kernel));
    if (e != cudaSuccess) return e;
    if (!g_bsms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_bsms, cudaDevAttrMultiProcessorCount, dev);
        if (!g_bsms) g_bsms = 148;
    }
    const int64_t grid = std::min<int64_t>(max_items, g_bsms);
    right_tc_batched_kernel<<<(unsigned)grid, kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace re
