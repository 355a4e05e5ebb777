// Right sketch A*X (Algorithm 1 step 3) for a Gaussian X on the 5th-generation
// tensor cores (tcgen05), with A split exactly into three BF16 terms:
//
//     a = hi + mid + lo,  hi = bf16(a), mid = bf16(a - hi), lo = bf16(a - hi - mid)
//
// (24 significand bits of FP32 in three 8-bit pieces; every step is exact in
// FP32), while X holds BF16-exact normals by construction, so each product is
// exact and only the FP32 accumulation rounds.  A*X = hi*X + mid*X + lo*X is
// accumulated in one TMEM accumulator.
//
// Persistent kernel, one CTA per SM, 128-row M tiles, K chunks of 64:
//   warps 0-7   converters: warp (q, h) reads, for row 32q + lane, the 32 FP32
//               values of half h of a chunk (conflict-free 16-byte loads of the
//               swizzled tile), splits them exactly into three BF16 terms and
//               writes them to TMEM (tcgen05.st, lanes 32q..32q+31), where the
//               MMA takes them as its A operand.  The split terms never touch
//               shared memory, which then carries only the TMA writes, the
//               converter reads and the MMA's reads of X^T.
//   warps 8-11  epilogue: tcgen05.ld (32 lanes x 16 columns) -> FP32 rows of AX.
//   warp 12     TMA producer of A: FP32 half chunks (128 rows x 32 k, 128B
//               swizzle, zero fill past the edges) into an 8 deep ring, so up
//               to 128 KB of A are in flight per SM.
//   warp 13     TMA producer of X^T: BF16 chunk (N rows x 64 k, 128B swizzle).
//   warp 14     TMEM allocation; one elected thread issues 3 x 4 tcgen05.mma
//               (M=128, N, K=16, kind::f16 BF16 -> FP32, A from TMEM) per chunk
//               and tcgen05.commit to release stages / publish accumulators.
// TMEM (512 columns): accumulators in [0, 256) -- double buffered for N <= 128
// so the epilogue of one tile overlaps the MMAs of the next -- and two A stages
// of 96 columns from column 256.  Every mbarrier wait is bounded in time: on
// expiry the kernel raises an error flag, every role drains what it has in
// flight (bounded again), TMEM is freed and the kernel returns.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

using namespace tc;

constexpr int kBM = 128;           // rows per M tile (UMMA M)
constexpr int kBK = 64;            // K elements per chunk (one 128-byte swizzle row)
constexpr int kConvParts = 1;                                  // converter warps per (lane quarter, half chunk); 2 measured slower
constexpr int kConvWarps = 8 * kConvParts;
constexpr int kEpiWarps = 4;
constexpr int kThreads = (kConvWarps + kEpiWarps + 3) * 32;
constexpr int kAProdWarp = kConvWarps + kEpiWarps;
constexpr int kBProdWarp = kAProdWarp + 1;
constexpr int kMmaWarp = kBProdWarp + 1;
constexpr int kHalfWarps = kConvWarps / 2;                     // converter warps per half chunk
constexpr uint32_t kHalfBytes = kBM * 32 * 4;                  // 16 KB FP32 half chunk
constexpr int kMaxAStages = 8;                                 // FP32 half-chunk ring depth
constexpr int kStages = 2;                                     // TMEM A stages = X^T stages
// TMEM columns: accumulators at [0, 256) (two N <= 128 buffers, or one N = 256),
// then kStages A stages of 3 terms x 32 columns (64 k of BF16 pairs)
constexpr uint32_t kAStageCol = 256;
constexpr uint32_t kTmemCols = 512;
static_assert(kAStageCol + 96 * kStages <= kTmemCols, "TMEM budget");

struct TcParams {
    const float* A;
    int64_t lda, M, K;
    float* C;
    int64_t ldc;
    int S;            // valid output columns
    int N;            // MMA N (>= 16, multiple of 16)
    int64_t tiles;
    int64_t kchunks;
    int* err;
    int drop_first;   // test hook: CTA 0 withholds its first A half chunk
    int xterms;       // BF16 planes of X (1: exact X; 2: X = hi + lo exactly; 3: FP32 X)
    int xrows;        // rows of one plane in the X^T map (plane t starts at row t * xrows)
};

// (A term, X term) products accumulated per K step with more than one plane of X
// (one plane: every A term times X): with two exact planes all six; with three planes the six whose terms
// carry at most 16 bits below the leading one (the rest are below 2^-24 relative).
__device__ constexpr int kPairs2A[6] = {0, 1, 2, 0, 1, 2}, kPairs2X[6] = {0, 0, 0, 1, 1, 1};
__device__ constexpr int kPairs3A[6] = {0, 0, 1, 0, 1, 2}, kPairs3X[6] = {0, 1, 0, 2, 1, 0};

__global__ void __launch_bounds__(kThreads, 1) right_tc_kernel(const __grid_constant__ CUtensorMap amap,
                                                               const __grid_constant__ CUtensorMap xmap,
                                                               const TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[kMaxAStages], a_empty[kMaxAStages];
    __shared__ __align__(8) uint64_t full_a[kStages], full_b[kStages], empty[kStages];
    __shared__ __align__(8) uint64_t accf[2], acce[2], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int NA = kMaxAStages;                  // compile time: ring indices are shifts
    const int nacc = p.N <= 128 ? 2 : 1;            // accumulator buffers in TMEM
    const uint32_t b_bytes = (uint32_t)p.N * kBK * 2;                 // one plane of one stage
    const uint32_t b_plane = (b_bytes + 1023u) & ~1023u;
    const uint32_t b_stage = b_plane * (uint32_t)p.xterms;
    unsigned char* abuf = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* bbuf = abuf + (size_t)NA * kHalfBytes;

    if (tid == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], kHalfWarps * 32);
        }
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full_a[i], kConvWarps * 32);
            mbar_init(&full_b[i], 1);
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

    // Stream-K schedule: the tiles x kchunks chunks (tile-major) are cut into
    // gridDim.x equal contiguous ranges; this CTA owns [c_begin, c_end).  A range
    // is never shorter than a tile (gridDim.x <= tiles), so a tile is shared by
    // at most two CTAs; both add their partial sums onto the zeroed output.
    const int64_t K = p.kchunks;
    const int64_t c_total = p.tiles * K;
    const int64_t c_begin = (int64_t)blockIdx.x * c_total / gridDim.x;
    const int64_t c_end = ((int64_t)blockIdx.x + 1) * c_total / gridDim.x;
    const int64_t total_chunks = c_end - c_begin;
    const int64_t t_first = c_begin / K;
    const int64_t nseg = total_chunks > 0 ? (c_end - 1) / K - t_first + 1 : 0;

    if (warp < kConvWarps) {
        // ---------------- converters: warp (q, h, part) owns TMEM lanes 32q.. (rows 32q + lane)
        // and k = 32h + (32 / kConvParts) part .. of every chunk: one FP32 row piece per thread.
        constexpr int KW = 32 / kConvParts;              // k per converter warp and chunk
        const int q = warp & 3, hp = warp >> 2, h = hp / kConvParts, part = hp % kConvParts;
        const int r = 32 * q + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        for (int64_t g = 0; g < total_chunks; ++g) {
            const int s = (int)(g % kStages);
            // the warp leaves together (tcgen05.st is a warp-wide instruction)
            bool ok = mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err);
            const int64_t hg = 2 * g + h;
            const int as = (int)(hg % NA);
            if (ok) ok = mbar_wait(&a_full[as], (uint32_t)((hg / NA) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;
            // row r of the 128B-swizzled half tile: 16-byte chunk c sits at slot c ^ (r & 7);
            // the 32 rows of a warp cover every bank four times per load (no conflicts)
            const unsigned char* src = abuf + (size_t)as * kHalfBytes + (size_t)r * 128;
            float4 v[KW / 4];
#pragma unroll
            for (int c = 0; c < KW / 4; ++c) {
                const int cc = (KW / 4) * part + c;
                v[c] = *reinterpret_cast<const float4*>(src + ((cc ^ (r & 7)) << 4));
            }
            mbar_arrive(&a_empty[as]);
            uint32_t hi[KW / 2], mid[KW / 2], lo[KW / 2];
#pragma unroll
            for (int c = 0; c < KW / 4; ++c) {
                split3(v[c].x, v[c].y, hi[2 * c], mid[2 * c], lo[2 * c]);
                split3(v[c].z, v[c].w, hi[2 * c + 1], mid[2 * c + 1], lo[2 * c + 1]);
            }
            tc_fence_after();
            // A operand layout in TMEM (M = 128): lane = row, 32-bit column = two
            // consecutive k (lower k in the low half); term t of stage s starts at
            // column kAStageCol + 96 s + 32 t, and k of this warp at +16 h + (KW / 2) part
            const uint32_t col = kAStageCol + 96u * (uint32_t)s + 16u * (uint32_t)h + (uint32_t)(KW / 2) * part;
            tmem_st<KW / 2>(lane_base + col, hi);
            tmem_st<KW / 2>(lane_base + col + 32u, mid);
            tmem_st<KW / 2>(lane_base + col + 64u, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&full_a[s]);
        }
    } else if (warp == kAProdWarp) {
        // ---------------- TMA producer of A half chunks
        if (lane == 0) {
            const bool drop0 = p.drop_first && blockIdx.x == 0;   // its converters' waits expire
            int64_t issued = 0;
            int64_t tile = c_begin / K, kc = c_begin % K;   // stepped, no division in the loop
            for (int64_t hg = 0; hg < 2 * total_chunks; ++hg) {
                const int as = (int)(hg % NA);
                if (!mbar_wait(&a_empty[as], (uint32_t)((hg / NA) & 1) ^ 1u, &s_abort, p.err)) break;
                // the converters read this stage through the generic proxy; order those
                // reads before the TMA (async proxy) overwrites it
                fence_proxy_async();
                if (!(drop0 && hg == 0)) {
                    mbar_arrive_expect_tx(&a_full[as], kHalfBytes);
                    tma_load_2d(abuf + (size_t)as * kHalfBytes, &amap, (int)(kc * kBK + 32 * (hg & 1)),
                                (int)(tile * kBM), &a_full[as]);
                }
                ++issued;
                if ((hg & 1) && ++kc == K) {
                    kc = 0;
                    ++tile;
                }
            }
            for (int64_t hg = std::max<int64_t>(0, issued - NA); hg < issued; ++hg)
                if (!(drop0 && hg == 0)) mbar_drain(&a_full[hg % NA], (uint32_t)((hg / NA) & 1));
        }
    } else if (warp == kBProdWarp) {
        // ---------------- TMA producer of X^T chunks
        if (lane == 0) {
            int64_t issued = 0;
            int64_t kc = c_begin % K;
            for (int64_t g = 0; g < total_chunks; ++g) {
                const int s = (int)(g % kStages);
                if (!mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err)) break;
                mbar_arrive_expect_tx(&full_b[s], b_bytes * (uint32_t)p.xterms);
                for (int t = 0; t < p.xterms; ++t)
                    tma_load_2d(bbuf + (size_t)s * b_stage + (size_t)t * b_plane, &xmap, (int)(kc * kBK), t * p.xrows,
                                &full_b[s]);
                ++issued;
                if (++kc == K) kc = 0;
            }
            for (int64_t g = std::max<int64_t>(0, issued - kStages); g < issued; ++g)
                mbar_drain(&full_b[g % kStages], (uint32_t)((g / kStages) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer: A terms from TMEM, X^T from shared memory
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(p.N);
            int64_t g = 0;
            bool ok = true;
            for (int64_t j = 0; j < nseg && ok; ++j) {
                const int a = (int)(j % nacc);
                if (!mbar_wait(&acce[a], (uint32_t)(((j / nacc) & 1) ^ 1), &s_abort, p.err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * p.N);
                const int64_t t0 = (t_first + j) * K;
                const int64_t k0 = std::max(c_begin, t0) - t0, k1 = std::min(c_end, t0 + K) - t0;
                for (int64_t kc = k0; kc < k1; ++kc, ++g) {
                    const int s = (int)(g % kStages);
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!mbar_wait(&full_a[s], ph, &s_abort, p.err) ||
                        !mbar_wait(&full_b[s], ph, &s_abort, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t bst = smem_u32(bbuf + (size_t)s * b_stage);
                    const uint32_t ast = tmem_base + kAStageCol + 96u * (uint32_t)s;
                    if (p.xterms == 1) {
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
                            const uint64_t bdesc = sw128_desc(bst + 32u * kk);
#pragma unroll
                            for (int term = 0; term < 3; ++term)
                                mma_bf16_ts(d_tmem, ast + 32u * term + 8u * kk, bdesc, idesc,
                                            (kc != k0 || kk || term) ? 1u : 0u);
                        }
                    } else {
                        const bool two = p.xterms == 2;
#pragma unroll
                        for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                            for (int pr = 0; pr < 6; ++pr) {
                                const int ta = two ? kPairs2A[pr] : kPairs3A[pr];
                                const int tx = two ? kPairs2X[pr] : kPairs3X[pr];
                                const uint64_t bdesc = sw128_desc(bst + (uint32_t)tx * b_plane + 32u * kk);
                                mma_bf16_ts(d_tmem, ast + 32u * ta + 8u * kk, bdesc, idesc,
                                            (kc != k0 || kk || pr) ? 1u : 0u);
                            }
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (ok) mma_commit(&accf[a]);
            }
            // all issued MMAs complete before TMEM is released
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    } else {
        // ---------------- epilogue warps: TMEM lanes 32*(warp%4) ..
        const int q = warp & 3;
        for (int64_t j = 0; j < nseg; ++j) {
            const int a = (int)(j % nacc);
            const bool ok = mbar_wait(&accf[a], (uint32_t)((j / nacc) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;   // tcgen05.ld is warp-wide
            tc_fence_after();
            const int64_t tile = t_first + j;
            // a tile shared with a neighbouring CTA: add onto the zeroed output (two
            // addends onto +0 give the same sum in either order)
            const bool shared = std::max(c_begin, tile * K) != tile * K || std::min(c_end, tile * K + K) != tile * K + K;
            const int64_t row = tile * kBM + q * 32 + lane;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * p.N);
            for (int c = 0; c < p.N; c += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c, v);
                if (row < p.M) {
                    float* dst = p.C + row * p.ldc + c;
#pragma unroll
                    for (int i = 0; i < 16; i += 4) {
                        if (c + i >= p.S) continue;
                        const float4 w = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
                        if (shared) atomicAdd(reinterpret_cast<float4*>(dst + i), w);
                        else *reinterpret_cast<float4*>(dst + i) = w;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[a]);
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

// Zero the output rows of every tile that two CTAs share (the tile holding the
// start of range b, b = 1 .. G-1, unless the range starts on a tile boundary).
__global__ void tc_zero_shared_tiles(float* __restrict__ C, int64_t ldc, int64_t M, int S, int64_t tiles,
                                     int64_t kchunks, int G) {
    const int64_t b = (int64_t)blockIdx.x + 1;
    const int64_t c = b * (tiles * kchunks) / G;
    if (c % kchunks == 0) return;
    const int64_t tile = c / kchunks;
    const int64_t r0 = tile * kBM;
    const int64_t rows = std::min<int64_t>(kBM, M - r0);
    const int q4 = S / 4;
    for (int64_t i = threadIdx.x; i < rows * q4; i += blockDim.x) {
        const int64_t r = r0 + i / q4;
        *reinterpret_cast<float4*>(C + r * ldc + 4 * (i % q4)) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// ---- host side --------------------------------------------------------------
int g_sms = 0;

}  // namespace

bool tc_supported(const MatView& A) {
    // FP32, not transposed, TMA-compatible (16-byte aligned base and row pitch),
    // at least one full tile in each dimension
    return A.dtype == RE_F32 && !A.trans && (A.ld % 4) == 0 && A.rows >= kBM && A.cols >= kBK &&
           (reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0 && encode_fn() != nullptr;
}

int tc_mma_n(int s) { return s <= 16 ? 16 : (s + 15) / 16 * 16; }

cudaError_t launch_right_tc(const MatView& A, const uint16_t* Xt, int64_t ldt, int s, float* C,
                            int64_t ldc, int* err_flag, cudaStream_t st, int* launches, int drop_first, int xterms) {
    if (s <= 0 || A.rows <= 0) return cudaSuccess;
    if (s > 256 || s % 8 != 0 || xterms < 1 || xterms > 3) return cudaErrorInvalidValue;
    const int N = tc_mma_n(s);
    if (xterms > 1 && N > 128) return cudaErrorInvalidValue;      // shared memory: three planes of 128 rows
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)ldt, (cuuint64_t)N * xterms};
    const cuuint64_t gstride[1] = {(cuuint64_t)ldt * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)N};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(Xt), gdim, gstride,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // A: FP32 (K, M) with row pitch ld; boxes of 32 k x 128 rows, zero fill past the edges
    CUtensorMap amap;
    const cuuint64_t adim[2] = {(cuuint64_t)A.cols, (cuuint64_t)A.rows};
    const cuuint64_t astride[1] = {(cuuint64_t)A.ld * 4};
    const cuuint32_t abox[2] = {32u, (cuuint32_t)kBM};
    r = enc(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A.ptr), adim, astride, abox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcParams p;
    p.A = static_cast<const float*>(A.ptr);
    p.lda = A.ld;
    p.M = A.rows;
    p.K = A.cols;
    p.C = C;
    p.ldc = ldc;
    p.S = s;
    p.N = N;
    p.tiles = (A.rows + kBM - 1) / kBM;
    p.kchunks = (A.cols + kBK - 1) / kBK;
    p.err = err_flag;
    p.drop_first = drop_first;
    p.xterms = xterms;
    p.xrows = N;
    const uint32_t b_bytes = (uint32_t)N * kBK * 2;
    const size_t smem =
        (size_t)kHalfBytes * kMaxAStages + ((b_bytes + 1023u) & ~1023u) * (size_t)xterms * kStages + 1024;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(right_tc_kernel));
    if (e != cudaSuccess) return e;
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t grid = std::min<int64_t>(p.tiles, g_sms);
    if (grid > 1 && p.tiles % grid != 0) {
        tc_zero_shared_tiles<<<(unsigned)(grid - 1), 256, 0, st>>>(C, ldc, A.rows, s, p.tiles, p.kchunks, (int)grid);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) ++*launches;
    }
    right_tc_kernel<<<(unsigned)grid, kThreads, smem, st>>>(amap, map, p);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace re
