// B = Q^T A (Algorithm 3 step 8, Sec. 5.1) on the 5th-generation tensor cores.
//
// Both factors are split exactly into three BF16 terms (a = hi + mid + lo, each
// step exact in FP32), and the six products whose terms carry at most 16 bits
// below the leading one are accumulated in FP32 in TMEM:
//
//     Q^T A ~ Qh Ah + Qh Am + Qm Ah + Qh Al + Qm Am + Ql Ah
//
// (the dropped Qm Al, Ql Am, Ql Al are below 2^-24 of |Q|^T |A|, the size of one
// FP32 rounding).  The output is computed transposed, B^T = A^T Q: one CTA owns
// 128 columns j of A (the UMMA M dimension) and up to 128 columns c of Q (N), and
// runs over one contiguous range of the rows i of A (the contraction); ranges
// are split across CTAs when the column tiles alone do not fill the GPU, their
// partial sums reduced afterwards in a fixed order.
//
//   warps 0-7   converters: warp (q, h) reads, for column 32q + lane of A, the 32
//               rows of half h of a 64-row chunk (one 4-byte load per row; a warp's
//               32 lanes read 128 consecutive bytes), splits consecutive row pairs
//               into packed BF16x2 terms and writes them to TMEM (tcgen05.st,
//               lanes 32q..), where the MMA takes them as its A operand.
//   warps 8-11  epilogue: tcgen05.ld (32 lanes x 16 columns) -> rows c of B (a
//               warp writes 32 consecutive j of one row: 128 contiguous bytes).
//   warp 12     TMA producer of A: 32 rows x 128 columns FP32 (no swizzle, zero
//               fill past the edges) into an 8 deep ring.
//   warp 13     TMA producer of Q^T: the three BF16 terms of a 64-row chunk (N
//               rows x 64 k each, 128-byte swizzle).
//   warp 14     TMEM allocation; one elected thread issues 6 x 4 tcgen05.mma
//               (M = 128, N, K = 16, kind::f16 BF16 -> FP32, A from TMEM) per chunk.
// Every mbarrier wait is bounded in time: on expiry the kernel raises an error
// flag, every role drains what it has in flight (bounded again), TMEM is freed
// and the kernel returns.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

using namespace tc;

constexpr int kBM = 128;                         // columns of A per tile (UMMA M)
constexpr int kBK = 64;                          // rows of A per chunk
constexpr int kNQ = 128;                         // columns of Q per launch (largest UMMA N here)
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = (kConvWarps + kEpiWarps + 3) * 32;
constexpr int kAProdWarp = kConvWarps + kEpiWarps;
constexpr int kBProdWarp = kAProdWarp + 1;
constexpr int kMmaWarp = kBProdWarp + 1;
constexpr uint32_t kHalfBytes = 32 * kBM * 4;    // 16 KB: 32 rows x 128 columns FP32
constexpr int kAStages = 8;                      // ring of A half chunks
constexpr int kStages = 2;                       // TMEM A stages = Q^T stages
constexpr uint32_t kTermBytes = kNQ * kBK * 2;   // 16 KB: one BF16 term of a Q^T chunk
constexpr uint32_t kAStageCol = 256;             // TMEM: accumulator at [0, N), A stages from 256
constexpr uint32_t kTmemCols = 512;
static_assert(kAStageCol + 96 * kStages <= kTmemCols, "TMEM budget");

struct QbTcParams {
    int64_t N;           // columns of A (output columns j)
    int64_t kchunks;     // 64-row chunks of A in all
    int64_t per;         // chunks per split
    int kq;              // valid Q columns in this launch
    int nmma;            // MMA N: kq rounded up to 16
    float* out;          // row c of the output at out + c * ldo (+ split * zstride)
    int64_t ldo;
    int64_t zstride;
    int* err;
};

// The six (A term, Q term) products kept, term 0 = hi, 1 = mid, 2 = lo.
__device__ constexpr int kPairA[6] = {0, 0, 1, 0, 1, 2};
__device__ constexpr int kPairQ[6] = {0, 1, 0, 2, 1, 0};

__global__ void __launch_bounds__(kThreads, 1) qb_product_tc_kernel(const __grid_constant__ CUtensorMap amap,
                                                                    const __grid_constant__ CUtensorMap qmap,
                                                                    const QbTcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[kAStages], a_empty[kAStages];
    __shared__ __align__(8) uint64_t full_a[kStages], full_b[kStages], empty[kStages];
    __shared__ __align__(8) uint64_t accf, done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t b_bytes = (uint32_t)p.nmma * kBK * 2;     // one term of one stage
    unsigned char* abuf = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* bbuf = abuf + (size_t)kAStages * kHalfBytes;
    constexpr uint32_t b_stage = 3 * kTermBytes;

    if (tid == 0) {
        for (int i = 0; i < kAStages; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], 4 * 32);                  // the four converter warps of one half
        }
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full_a[i], kConvWarps * 32);
            mbar_init(&full_b[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accf, 1);
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

    const int64_t j0 = (int64_t)blockIdx.x * kBM;
    const int64_t c_begin = (int64_t)blockIdx.y * p.per;
    const int64_t c_end = std::min(p.kchunks, c_begin + p.per);
    const int64_t nch = c_end > c_begin ? c_end - c_begin : 0;

    if (warp < kConvWarps) {
        // ---------------- converters: warp (q, h) owns TMEM lanes 32q.. (columns j0 + 32q + lane)
        // and rows 32h .. 32h + 31 of every chunk
        const int q = warp & 3, h = warp >> 2;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        for (int64_t g = 0; g < nch; ++g) {
            const int s = (int)(g % kStages);
            bool ok = mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err);
            const int64_t hg = 2 * g + h;
            const int as = (int)(hg % kAStages);
            if (ok) ok = mbar_wait(&a_full[as], (uint32_t)((hg / kAStages) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;
            const float* src = reinterpret_cast<const float*>(abuf + (size_t)as * kHalfBytes) + 32 * q + lane;
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = src[i * kBM];
            mbar_arrive(&a_empty[as]);
            uint32_t hi[16], mid[16], lo[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) split3(v[2 * c], v[2 * c + 1], hi[c], mid[c], lo[c]);
            tc_fence_after();
            // A operand in TMEM (M = 128): lane = column j, 32-bit column = two consecutive
            // rows i (lower row in the low half); term t of stage s at kAStageCol + 96 s + 32 t
            const uint32_t col = kAStageCol + 96u * (uint32_t)s + 16u * (uint32_t)h;
            tmem_st16(lane_base + col, hi);
            tmem_st16(lane_base + col + 32u, mid);
            tmem_st16(lane_base + col + 64u, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&full_a[s]);
        }
    } else if (warp == kAProdWarp) {
        // ---------------- TMA producer of A half chunks (32 rows x 128 columns)
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t hg = 0; hg < 2 * nch; ++hg) {
                const int as = (int)(hg % kAStages);
                if (!mbar_wait(&a_empty[as], (uint32_t)((hg / kAStages) & 1) ^ 1u, &s_abort, p.err)) break;
                // the converters read this stage through the generic proxy; order those
                // reads before the TMA (async proxy) overwrites it
                fence_proxy_async();
                mbar_arrive_expect_tx(&a_full[as], kHalfBytes);
                tma_load_2d(abuf + (size_t)as * kHalfBytes, &amap, (int)j0,
                            (int)((c_begin + hg / 2) * kBK + 32 * (hg & 1)), &a_full[as]);
                ++issued;
            }
            for (int64_t hg = std::max<int64_t>(0, issued - kAStages); hg < issued; ++hg)
                mbar_drain(&a_full[hg % kAStages], (uint32_t)((hg / kAStages) & 1));
        }
    } else if (warp == kBProdWarp) {
        // ---------------- TMA producer of the three Q^T terms of a chunk
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t g = 0; g < nch; ++g) {
                const int s = (int)(g % kStages);
                if (!mbar_wait(&empty[s], (uint32_t)((g / kStages) & 1) ^ 1u, &s_abort, p.err)) break;
                mbar_arrive_expect_tx(&full_b[s], 3 * b_bytes);
#pragma unroll
                for (int t = 0; t < 3; ++t)
                    tma_load_3d(bbuf + (size_t)s * b_stage + (size_t)t * kTermBytes, &qmap,
                                (int)((c_begin + g) * kBK), 0, t, &full_b[s]);
                ++issued;
            }
            for (int64_t g = std::max<int64_t>(0, issued - kStages); g < issued; ++g)
                mbar_drain(&full_b[g % kStages], (uint32_t)((g / kStages) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer: A terms from TMEM, Q^T terms from shared memory
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(p.nmma);
            bool ok = true;
            for (int64_t g = 0; g < nch && ok; ++g) {
                const int s = (int)(g % kStages);
                const uint32_t ph = (uint32_t)((g / kStages) & 1);
                if (!mbar_wait(&full_a[s], ph, &s_abort, p.err) || !mbar_wait(&full_b[s], ph, &s_abort, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t bst = smem_u32(bbuf + (size_t)s * b_stage);
                const uint32_t ast = tmem_base + kAStageCol + 96u * (uint32_t)s;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
#pragma unroll
                    for (int pr = 0; pr < 6; ++pr) {
                        const uint64_t bdesc = sw128_desc(bst + (uint32_t)kPairQ[pr] * kTermBytes + 32u * kk);
                        mma_bf16_ts(tmem_base, ast + 32u * kPairA[pr] + 8u * kk, bdesc, idesc,
                                    (g || kk || pr) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[s]);
            }
            if (ok) mma_commit(&accf);
            // all issued MMAs complete before TMEM is released
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    } else {
        // ---------------- epilogue warps: TMEM lanes 32 (warp % 4) ..
        const int q = warp & 3;
        const bool ok = nch > 0 && mbar_wait(&accf, 0, &s_abort, p.err);
        if (__all_sync(0xffffffffu, ok)) {
            tc_fence_after();
            const int64_t j = j0 + q * 32 + lane;
            float* out = p.out + (int64_t)blockIdx.y * p.zstride;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16);
            for (int c = 0; c < p.nmma; c += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c, v);
                if (j < p.N) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c + i < p.kq) out[(int64_t)(c + i) * p.ldo + j] = v[i];
                }
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

// Qt[t][c][i] (BF16 bits, row pitch ldt, `rows` rows per term) = term t of
// Q[i][c] for c < k, 0 for k <= c < rows; i < M.  32 x 32 tiles through shared
// memory so that both the reads (along c) and the writes (along i) are coalesced.
__global__ void qt_split_kernel(const float* __restrict__ Q, int64_t ldq, int64_t M, int k, int rows,
                                uint16_t* __restrict__ Qt, int64_t ldt) {
    __shared__ float T[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = i0 + r;
        const int c = c0 + (int)threadIdx.x;
        T[r][threadIdx.x] = (i < M && c < k) ? Q[i * ldq + c] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r;
        const int64_t i = i0 + threadIdx.x;
        if (c >= rows || i >= M) continue;
        const float a = T[threadIdx.x][r];
        uint32_t hi, mid, lo;
        split3(a, 0.f, hi, mid, lo);      // the low halves hold the terms of a
        const int64_t o = (int64_t)c * ldt + i;
        Qt[o] = (uint16_t)(hi & 0xFFFFu);
        Qt[(int64_t)rows * ldt + o] = (uint16_t)(mid & 0xFFFFu);
        Qt[(int64_t)2 * rows * ldt + o] = (uint16_t)(lo & 0xFFFFu);
    }
}

int g_sms = 0;

}  // namespace

bool qb_tc_supported(const MatView& A) {
    // FP32, not transposed, TMA-compatible rows (16-byte aligned base and pitch)
    return A.dtype == RE_F32 && !A.trans && (A.ld % 4) == 0 && (reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0 &&
           encode_fn() != nullptr;
}

int64_t qb_tc_qt_ld(int64_t M) { return (M + 7) / 8 * 8; }

int qb_tc_qt_rows(int k) { return (k + kNQ - 1) / kNQ * kNQ; }

// Split count for `tiles` column tiles: the fewest splits (at most cap, at least
// 8 chunks each) whose CTAs fill whole waves of the SMs best.
int qb_tc_splits(int64_t tiles, int64_t kchunks, int cap) {
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_sms <= 0) g_sms = 1;
    }
    int best = 1;
    double best_eff = 0.0;
    const int64_t smax = std::max<int64_t>(1, std::min<int64_t>(cap, kchunks / 8));
    for (int64_t s = 1; s <= smax; ++s) {
        const int64_t ctas = tiles * s;
        const int64_t waves = (ctas + g_sms - 1) / g_sms;
        const double eff = (double)ctas / (double)(waves * g_sms);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = (int)s;
        }
    }
    return best;
}

cudaError_t launch_qt_split(const float* Q, int64_t ldq, int64_t M, int k, uint16_t* Qt, cudaStream_t st) {
    const int rows = qb_tc_qt_rows(k);
    const dim3 grid((unsigned)((M + 31) / 32), (unsigned)(rows / 32));
    qt_split_kernel<<<grid, dim3(32, 8), 0, st>>>(Q, ldq, M, k, rows, Qt, qb_tc_qt_ld(M));
    return cudaGetLastError();
}

// Columns [c0, c0 + kq) of Q (kq <= 128): out (row c - c0 at out + (c - c0) ldo, or
// the split partials at part + z zstride with pitch N) = (Q^T A)[c][:].
cudaError_t launch_qb_product_tc(const MatView& A, const uint16_t* Qt, int k, int c0, int kq, float* out,
                                 int64_t ldo, float* part, int splits, int* err_flag, cudaStream_t st,
                                 double* out64, int64_t ldo64) {
    if (kq <= 0 || kq > kNQ) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int64_t M = A.rows, N = A.cols;
    const int nmma = (kq + 15) / 16 * 16;
    const int rows = qb_tc_qt_rows(k);
    const int64_t ldt = qb_tc_qt_ld(M);
    // Q^T terms: a 3-D BF16 map (row i, column c from c0, term t) over Qt, whose term t
    // of column c sits at row t * rows + c (pitch ldt); boxes of 64 rows x nmma columns
    // x 1 term, 128-byte swizzle (one 128-byte line per column and 64-row chunk)
    CUtensorMap qmap;
    const cuuint64_t qdim[3] = {(cuuint64_t)M, (cuuint64_t)nmma, 3};
    const cuuint64_t qstride[2] = {(cuuint64_t)ldt * 2, (cuuint64_t)ldt * 2 * rows};
    const cuuint32_t qbox[3] = {(cuuint32_t)kBK, (cuuint32_t)nmma, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&qmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<uint16_t*>(Qt) + (size_t)c0 * ldt,
                     qdim, qstride, qbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // A: FP32 (N columns, M rows) with row pitch ld; boxes of 128 columns x 32 rows, no
    // swizzle, zero fill past the edges
    CUtensorMap amap;
    const cuuint64_t adim[2] = {(cuuint64_t)N, (cuuint64_t)M};
    const cuuint64_t astride[1] = {(cuuint64_t)A.ld * 4};
    const cuuint32_t abox[2] = {(cuuint32_t)kBM, 32u};
    r = enc(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A.ptr), adim, astride, abox, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    QbTcParams p;
    p.N = N;
    p.kchunks = (M + kBK - 1) / kBK;
    p.per = (p.kchunks + splits - 1) / splits;
    const int used = (int)((p.kchunks + p.per - 1) / p.per);     // splits that own at least one chunk
    p.kq = kq;
    p.nmma = nmma;
    // an FP64 output always takes the partials (one or more) and the FP64 reduction
    const bool parts = splits > 1 || out64 != nullptr;
    p.out = parts ? part : out;
    p.ldo = parts ? N : ldo;
    p.zstride = (int64_t)kq * N;
    p.err = err_flag;
    const size_t smem = (size_t)kHalfBytes * kAStages + (size_t)3 * kTermBytes * kStages + 1024;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(qb_product_tc_kernel));
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((N + kBM - 1) / kBM), (unsigned)used);
    qb_product_tc_kernel<<<grid, kThreads, smem, st>>>(amap, qmap, p);
    e = cudaGetLastError();
    if (e != cudaSuccess || !parts) return e;
    // splits that own no chunk leave their partial unwritten: the reduction covers `used`
    if (out64) return reduce_parts_f64(part, used, (int64_t)kq, N, out64, ldo64, st);
    return reduce_parts_f32(part, used, (int64_t)kq, N, out, ldo, st);
}

namespace {
// Plane t, row j (j < nrows), column l (l < ldt) of the X^T operand of the
// tensor-core right sketch for X = S^T, S rows c0 .. c0+w-1 (FP32, pitch lds,
// cols columns): term t of S[c0 + j][l], zero past w rows or cols columns.
__global__ void rows_split3_kernel(const float* __restrict__ S, int64_t lds, int c0, int w, int cols, int nrows,
                                   int64_t ldt, uint16_t* __restrict__ Xt) {
    const int64_t total = (int64_t)nrows * ldt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i / ldt);
        const int l = (int)(i - (int64_t)j * ldt);
        const float v = (j < w && l < cols) ? S[(int64_t)(c0 + j) * lds + l] : 0.f;
        uint32_t hi, mid, lo;
        split3(v, 0.f, hi, mid, lo);                   // the low halves hold the terms of v
        Xt[i] = (uint16_t)(hi & 0xffffu);
        Xt[total + i] = (uint16_t)(mid & 0xffffu);
        Xt[2 * total + i] = (uint16_t)(lo & 0xffffu);
    }
}
}  // namespace

cudaError_t launch_rows_split3(const float* S, int64_t lds, int c0, int w, int cols, int nrows, int64_t ldt,
                               uint16_t* Xt, cudaStream_t st) {
    if (w <= 0 || w > nrows || cols <= 0 || cols > ldt) return cudaErrorInvalidValue;
    const int64_t total = (int64_t)nrows * ldt;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 2048);
    rows_split3_kernel<<<blocks, 256, 0, st>>>(S, lds, c0, w, cols, nrows, ldt, Xt);
    return cudaGetLastError();
}

}  // namespace re
