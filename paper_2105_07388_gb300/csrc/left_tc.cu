// Left sketch on the tensor cores (Algorithm 1 steps 4-6 for a Gaussian or an
// SRCT Y): a block of the core Y (AX), computed transposed so that AX is the MMA's A
// operand.  For an M tile of 128 AX columns c, an N tile of up to 256 Y rows q
// and a range of AX rows i (split-K):
//
//     D[c][q] = sum_i AX[i][c] Y[q][i]
//
// AX (FP32) is split exactly into three BF16 terms (as in the right sketch) and
// written to TMEM; the entries of Y are BF16-exact normals, generated on the fly
// from Philox straight into the 128B-swizzled K-major layout of the B operand
// (Y never exists in HBM).  Products are exact; the FP32 accumulation in TMEM is
// the only rounding.  Each CTA writes its FP32 partial block, and the split-K
// partials are summed in FP64 in a fixed order afterwards.
//
// SRCT Y (the DCT-II rows of the sampled frequencies, Sec. 4 with eta = 2): an
// entry d_i sqrt(2) cos(pi (2i+1) k / 2N) is an FP32 value from the cosine table,
// so it enters as its three exact BF16 terms (three B planes per stage) and six
// products are issued per K step, the pairs of A and Y terms whose indices sum to
// at most 2 (as the three-plane right sketch).  N is at most 128 there, so that
// three planes of two stages fit in shared memory.
//
// Warp roles (576 threads, one CTA per SM):
//   warps 0-15   workers: for each 64-row chunk, warp w first generates its
//                share of Y (groups of 4 Y rows x 64 i: lane l makes the 2 Philox
//                calls of i = 2l, 2l+1 and writes one 4-byte word per row), then
//                converts 16 rows of AX for the TMEM lanes 32 (w & 3) .. (AX
//                columns of the M tile): loads of the row-major tile, exact split,
//                three tcgen05.st of 8 columns; warps 0-3 then run the epilogue.
//   warp 16      TMA producer of AX half chunks (32 rows x up to 128 columns,
//                FP32, zero fill past the last row / column).
//   warp 17      TMEM allocation and the MMA issuer (A from TMEM, B from smem).
// Every mbarrier wait is bounded in time (on expiry: error flag, drain, free
// TMEM, return).
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

using namespace tc;

constexpr int kLBM = 128;                    // AX columns per M tile (TMEM lanes)
constexpr int kLBK = 64;                     // AX rows per chunk
constexpr int kLWork = 16;                   // worker warps 0-15
constexpr int kLProdWarp = kLWork;           // 16
constexpr int kLMmaWarp = kLProdWarp + 1;    // 17
constexpr int kLThreads = (kLMmaWarp + 1) * 32;
constexpr int kLAStages = 4;                 // FP32 half-chunk ring
constexpr int kLStages = 2;                  // TMEM A stages = Y stages
constexpr uint32_t kLAStageCol = 256;        // TMEM: D in [0, N), A stages from column 256
constexpr uint32_t kLTmemCols = 512;
static_assert(kLAStageCol + 96 * kLStages <= kLTmemCols, "TMEM budget");

struct LeftTcParams {
    uint64_t seed;
    DctRows dct;        // SRCT rows (DCT mode only)
    int64_t M;          // AX rows
    int row0;           // first Y row of the block (a multiple of 4)
    int R;              // Y rows in the block
    int S;              // AX columns in the block
    int boxw;           // AX columns per TMA box (min(128, S))
    int N;              // MMA N (multiple of 16, <= 256)
    int n_tiles, m_tiles, splits;
    int64_t chunk;      // AX rows per split (a multiple of 64)
    float* part;        // [splits][R][S]
    int* err;
};

// Entry (q, i) of the SRCT left embedding from its row frequency k and sign d: the
// phase (2i+1) k is reduced modulo 4N (4N divides 2^32, so the wrapped 32-bit
// product has the right residue) and folded onto [0, N].
__device__ __forceinline__ float dct_y_entry(const DctRows& Y, uint32_t k, uint32_t i, float d) {
    if (k == 0) return d;
    const uint32_t N = 1u << Y.nbits, twoN = 2u * N, fourN = 4u * N;
    uint32_t ph = ((2u * i + 1u) * k) & (fourN - 1u);
    if (ph > twoN) ph = fourN - ph;
    const float c = ph <= N ? __ldg(Y.ctab + ph) : -__ldg(Y.ctab + (twoN - ph));
    return 1.41421356237309515f * c * d;
}

template <bool DCT>
__global__ void __launch_bounds__(kLThreads, 1) left_tc_kernel(const __grid_constant__ CUtensorMap amap,
                                                               const LeftTcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[kLAStages], a_empty[kLAStages];
    __shared__ __align__(8) uint64_t full[kLStages], empty[kLStages];
    __shared__ __align__(8) uint64_t accf, done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = p.n_tiles * p.m_tiles;
    const int split = blockIdx.x / tiles;
    const int nt = (blockIdx.x % tiles) / p.m_tiles;
    const int mt = blockIdx.x % p.m_tiles;
    const int64_t i_begin = (int64_t)split * p.chunk;
    const int64_t i_end = std::min<int64_t>(p.M, i_begin + p.chunk);
    const int64_t nchunks = i_end > i_begin ? (i_end - i_begin + kLBK - 1) / kLBK : 0;
    const uint32_t half_bytes = (uint32_t)p.boxw * 32u * 4u;
    constexpr int kYTerms = DCT ? 3 : 1;
    const uint32_t y_plane = ((uint32_t)p.N * 128u + 1023u) & ~1023u;
    const uint32_t y_stage = y_plane * (uint32_t)kYTerms;
    unsigned char* abuf = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* ybuf = abuf + (size_t)kLAStages * ((kLBM * 32 * 4 + 1023) & ~1023);

    if (tid == 0) {
        for (int i = 0; i < kLAStages; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], (kLWork / 2) * 32);
        }
        for (int i = 0; i < kLStages; ++i) {
            mbar_init(&full[i], kLWork * 32);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accf, 1);
        mbar_init(&done_bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    if (warp == kLMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(kLTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem;

    if (warp < kLWork) {
        // ---------------- workers
        const int q = warp & 3, r4 = warp >> 2;        // TMEM lane quarter, 16-row quarter of a chunk
        const int h = r4 >> 1, roff = (r4 & 1) * 16;   // A half holding those rows, offset inside it
        const int c = 32 * q + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(32 * q) << 16);
        const int rows_here = std::min(p.N, p.R - nt * p.N);
        const uint32_t q4_base = (uint32_t)((p.row0 + nt * p.N) >> 2);
        const int chunk16 = lane >> 2;                 // 16-byte segment of a Y row
        const uint32_t in_seg = (uint32_t)(lane & 3) * 4u;
        for (int64_t g = 0; g < nchunks; ++g) {
            const int s = (int)(g % kLStages);
            bool ok = mbar_wait(&empty[s], (uint32_t)((g / kLStages) & 1) ^ 1u, &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;
            // Y share: groups of 4 rows
            unsigned char* yb = ybuf + (size_t)s * y_stage;
            const int64_t i0 = i_begin + g * kLBK + 2 * lane;
            if constexpr (DCT) {
                // one row per step: lane l forms the entries i0 = 2l, 2l+1 of the chunk
                const uint32_t db = i0 < p.M ? __ldg(p.dct.dbits + (i0 >> 5)) : 0u;   // i0 even: one word
                const float d0 = ((db >> (i0 & 31)) & 1u) ? -1.f : 1.f;
                const float d1 = ((db >> ((i0 + 1) & 31)) & 1u) ? -1.f : 1.f;
                const int qrow = p.row0 + nt * p.N;
                for (int ql = warp; ql < p.N; ql += kLWork) {
                    uint32_t wh = 0u, wm = 0u, wl = 0u;
                    if (ql < rows_here) {
                        const uint32_t k = (uint32_t)__ldg(p.dct.krow + qrow + ql);
                        const float e0 = i0 < p.M ? dct_y_entry(p.dct, k, (uint32_t)i0, d0) : 0.f;
                        const float e1 = i0 + 1 < p.M ? dct_y_entry(p.dct, k, (uint32_t)(i0 + 1), d1) : 0.f;
                        split3(e0, e1, wh, wm, wl);
                    }
                    const size_t off = (size_t)ql * 128 + ((chunk16 ^ (ql & 7)) << 4) + in_seg;
                    *reinterpret_cast<uint32_t*>(yb + off) = wh;
                    *reinterpret_cast<uint32_t*>(yb + y_plane + off) = wm;
                    *reinterpret_cast<uint32_t*>(yb + 2 * (size_t)y_plane + off) = wl;
                }
            } else {
                for (int grp = warp; grp < p.N / 4; grp += kLWork) {
                    float z0[4], z1[4];
                    if (4 * grp < rows_here && i0 < p.M) {
                        normals4((uint32_t)i0, q4_base + (uint32_t)grp, kStreamGY, p.seed, z0);
                    } else {
                        z0[0] = z0[1] = z0[2] = z0[3] = 0.f;
                    }
                    if (4 * grp < rows_here && i0 + 1 < p.M) {
                        normals4((uint32_t)(i0 + 1), q4_base + (uint32_t)grp, kStreamGY, p.seed, z1);
                    } else {
                        z1[0] = z1[1] = z1[2] = z1[3] = 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int ql = 4 * grp + e;
                        const uint32_t w = ql < rows_here
                                               ? ((__float_as_uint(z0[e]) >> 16) | (__float_as_uint(z1[e]) & 0xFFFF0000u))
                                               : 0u;
                        *reinterpret_cast<uint32_t*>(yb + (size_t)ql * 128 + ((chunk16 ^ (ql & 7)) << 4) + in_seg) = w;
                    }
                }
            }
            fence_proxy_async();
            // AX share: rows roff .. roff+15 of half h, column c
            const int64_t hg = 2 * g + h;
            const int as = (int)(hg % kLAStages);
            ok = mbar_wait(&a_full[as], (uint32_t)((hg / kLAStages) & 1), &s_abort, p.err);
            if (!__all_sync(0xffffffffu, ok)) break;     // tcgen05.st is warp-wide
            const float* src = reinterpret_cast<const float*>(abuf + (size_t)as * ((kLBM * 32 * 4 + 1023) & ~1023));
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = c < p.boxw ? src[(roff + i) * p.boxw + c] : 0.f;
            mbar_arrive(&a_empty[as]);
            uint32_t hi[8], mid[8], lo[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) split3(v[2 * i], v[2 * i + 1], hi[i], mid[i], lo[i]);
            tc_fence_after();
            // A stage layout: term t at column kLAStageCol + 96 s + 32 t, K pair k/2 at +k/2
            const uint32_t col = kLAStageCol + 96u * (uint32_t)s + 8u * (uint32_t)r4;
            tmem_st8(lane_base + col, hi);
            tmem_st8(lane_base + col + 32u, mid);
            tmem_st8(lane_base + col + 64u, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            mbar_arrive(&full[s]);
        }
        if (warp < 4) {
            // ---------------- epilogue: lane c of the M tile, N columns of D
            const bool done = nchunks > 0 && mbar_wait(&accf, 0u, &s_abort, p.err);
            if (__all_sync(0xffffffffu, done)) {
                tc_fence_after();
                const int cg = mt * kLBM + c;
                for (int col = 0; col < p.N; col += 16) {
                    float v[16];
                    tmem_ld16(lane_base + (uint32_t)col, v);
                    if (cg < p.S) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int r = nt * p.N + col + u;
                            if (r < p.R) p.part[((int64_t)split * p.R + r) * p.S + cg] = v[u];
                        }
                    }
                }
            }
        }
    } else if (warp == kLProdWarp) {
        // ---------------- TMA producer of AX half chunks
        if (lane == 0) {
            const uint32_t a_stage = (kLBM * 32 * 4 + 1023) & ~1023;
            int64_t issued = 0;
            for (int64_t hg = 0; hg < 2 * nchunks; ++hg) {
                const int as = (int)(hg % kLAStages);
                if (!mbar_wait(&a_empty[as], (uint32_t)((hg / kLAStages) & 1) ^ 1u, &s_abort, p.err)) break;
                // the workers read this stage through the generic proxy; order those reads
                // before the TMA (async proxy) overwrites it
                fence_proxy_async();
                mbar_arrive_expect_tx(&a_full[as], half_bytes);
                tma_load_2d(abuf + (size_t)as * a_stage, &amap, mt * kLBM, (int)(i_begin + 32 * hg), &a_full[as]);
                ++issued;
            }
            for (int64_t hg = std::max<int64_t>(0, issued - kLAStages); hg < issued; ++hg)
                mbar_drain(&a_full[hg % kLAStages], (uint32_t)((hg / kLAStages) & 1));
        }
    } else {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(p.N);
            bool ok = true;
            for (int64_t g = 0; g < nchunks; ++g) {
                const int s = (int)(g % kLStages);
                const uint32_t ph = (uint32_t)((g / kLStages) & 1);
                if (!mbar_wait(&full[s], ph, &s_abort, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t bst = smem_u32(ybuf + (size_t)s * y_stage);
                const uint32_t ast = tmem_base + kLAStageCol + 96u * (uint32_t)s;
#pragma unroll
                for (int kk = 0; kk < kLBK / 16; ++kk) {
                    if constexpr (DCT) {
                        // AX term ta with Y term ty, ta + ty <= 2
                        constexpr int kTa[6] = {0, 0, 1, 0, 1, 2}, kTy[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
                        for (int pr = 0; pr < 6; ++pr) {
                            const uint64_t bdesc = sw128_desc(bst + (uint32_t)kTy[pr] * y_plane + 32u * kk);
                            mma_bf16_ts(tmem_base, ast + 32u * kTa[pr] + 8u * kk, bdesc, idesc,
                                        (g | kk | pr) ? 1u : 0u);
                        }
                    } else {
                        const uint64_t bdesc = sw128_desc(bst + 32u * kk);
#pragma unroll
                        for (int term = 0; term < 3; ++term)
                            mma_bf16_ts(tmem_base, ast + 32u * term + 8u * kk, bdesc, idesc,
                                        (g | kk | term) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[s]);
            }
            if (ok && nchunks > 0) mma_commit(&accf);
            mma_commit(&done_bar);
            mbar_drain(&done_bar, 0);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kLMmaWarp) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kLTmemCols)
                     : "memory");
    }
}

int g_left_sms = 0;

int left_sms() {
    if (!g_left_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_left_sms, cudaDevAttrMultiProcessorCount, dev);
        if (!g_left_sms) g_left_sms = 148;
    }
    return g_left_sms;
}

struct LeftTcPlan {
    int N, n_tiles, m_tiles, splits;
    int64_t chunk;
};

LeftTcPlan left_tc_plan(int64_t M, int R, int S, size_t part_cap, bool dct) {
    LeftTcPlan pl;
    pl.N = std::min(dct ? 128 : 256, (R + 15) / 16 * 16);
    pl.n_tiles = (R + pl.N - 1) / pl.N;
    pl.m_tiles = (S + kLBM - 1) / kLBM;
    const int tiles = pl.n_tiles * pl.m_tiles;
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>((M + kLBK - 1) / kLBK, (left_sms() + tiles - 1) / tiles));
    if (part_cap > 0) splits = std::min<int64_t>(splits, (int64_t)(part_cap / ((size_t)R * S)));
    splits = std::max<int64_t>(splits, 1);
    int64_t chunk = (M + splits - 1) / splits;
    chunk = (chunk + kLBK - 1) / kLBK * kLBK;
    pl.chunk = chunk;
    pl.splits = (int)((M + chunk - 1) / chunk);
    return pl;
}

}  // namespace

bool left_tc_supported(const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0, int S) {
    return encode_fn() != nullptr && M >= 32 && R >= 1 && S >= 4 && (S % 4) == 0 && (row0 % 4) == 0 &&
           (ldax % 4) == 0 && (reinterpret_cast<uintptr_t>(AX + col0) & 15) == 0;
}

size_t left_tc_part_floats(int64_t M, int R, int S, bool dct) {
    const LeftTcPlan pl = left_tc_plan(M, R, S, 0, dct);
    return (size_t)pl.splits * R * S;
}

cudaError_t launch_left_tc_partials(uint64_t seed, const float* AX, int64_t ldax, int64_t M, int row0, int R,
                                    int col0, int S, float* part, size_t part_cap, int* err_flag, int* splits_out,
                                    cudaStream_t st, const DctRows* dct) {
    const bool is_dct = dct != nullptr;
    if (is_dct && (dct->nbits < 0 || dct->nbits > 29 || (M > (int64_t(1) << dct->nbits)))) return cudaErrorInvalidValue;
    const LeftTcPlan pl = left_tc_plan(M, R, S, part_cap, is_dct);
    if ((size_t)pl.splits * R * S > part_cap) return cudaErrorInvalidValue;
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int boxw = std::min(kLBM, S);
    CUtensorMap amap;
    const cuuint64_t dim[2] = {(cuuint64_t)S, (cuuint64_t)M};
    const cuuint64_t stride[1] = {(cuuint64_t)ldax * 4};
    const cuuint32_t box[2] = {(cuuint32_t)boxw, 32u};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(AX + col0), dim, stride, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    LeftTcParams p;
    p.seed = seed;
    p.dct = is_dct ? *dct : DctRows{nullptr, nullptr, nullptr, 0};
    p.M = M;
    p.row0 = row0;
    p.R = R;
    p.S = S;
    p.boxw = boxw;
    p.N = pl.N;
    p.n_tiles = pl.n_tiles;
    p.m_tiles = pl.m_tiles;
    p.splits = pl.splits;
    p.chunk = pl.chunk;
    p.part = part;
    p.err = err_flag;
    const size_t a_stage = (kLBM * 32 * 4 + 1023) & ~1023;
    const size_t y_stage = (((size_t)pl.N * 128 + 1023) & ~(size_t)1023) * (is_dct ? 3 : 1);
    const size_t smem = a_stage * kLAStages + y_stage * kLStages + 1024;
    const void* kern = is_dct ? reinterpret_cast<const void*>(left_tc_kernel<true>)
                              : reinterpret_cast<const void*>(left_tc_kernel<false>);
    cudaError_t e = allow_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    const int64_t grid = (int64_t)pl.splits * pl.n_tiles * pl.m_tiles;
    if (grid > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (is_dct)
        left_tc_kernel<true><<<(unsigned)grid, kLThreads, smem, st>>>(amap, p);
    else
        left_tc_kernel<false><<<(unsigned)grid, kLThreads, smem, st>>>(amap, p);
    *splits_out = pl.splits;
    return cudaGetLastError();
}

}  // namespace re
