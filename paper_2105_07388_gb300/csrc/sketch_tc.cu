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
//   warp 12     TMA producer of A: FP32 half chunks (128 rows x 32 k, 128B
//               swizzle, zero fill past the edges) into a 3-4 deep ring, so
//               48-64 KB of A are in flight per SM.
//   warp 13     TMA producer of X^T: BF16 chunk (N rows x 64 k, 128B swizzle).
//   warps 0-7   converters: read two FP32 half chunks from shared memory, split
//               exactly into three BF16 tiles written in the 128B-swizzled
//               K-major layout of the MMA descriptors; fence.proxy.async, arrive.
//   warp 14     TMEM allocation; one elected thread issues 3 x 4 tcgen05.mma
//               (M=128, N, K=16, kind::f16 BF16 -> FP32) per chunk and
//               tcgen05.commit to release stages / publish accumulators.
//   warps 8-11  epilogue: tcgen05.ld (32 lanes x 16 columns) -> FP32 rows of AX.
// The accumulator is double buffered in TMEM (2N columns) so the epilogue of one
// tile overlaps the MMAs of the next.  Every mbarrier wait is bounded in time:
// on expiry the kernel raises an error flag, every role drains what it has in
// flight (bounded again), TMEM is freed and the kernel returns.
#include <cuda.h>

#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kBM = 128;           // rows per M tile (UMMA M)
constexpr int kBK = 64;            // K elements per chunk (one 128-byte swizzle row)
constexpr int kConvWarps = 8;
constexpr int kEpiWarps = 4;
constexpr int kThreads = (kConvWarps + kEpiWarps + 3) * 32;   // 480
constexpr int kAProdWarp = kConvWarps + kEpiWarps;             // 12
constexpr int kBProdWarp = kAProdWarp + 1;                     // 13
constexpr int kMmaWarp = kBProdWarp + 1;                       // 14
constexpr uint32_t kTermBytes = kBM * kBK * 2;                 // 16 KB per BF16 term tile
constexpr uint32_t kHalfBytes = kBM * 32 * 4;                  // 16 KB FP32 half chunk
constexpr int kSplitStages = 2;
constexpr unsigned long long kWaitNs = 2000000000ull;          // 2 s bound per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the abort flag) on expiry or when
// another role has already aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (true) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_flag) return false;
        if (now_ns() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
}

// Wait used while draining after an abort: bounded, never raises anything.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = now_ns();
    while (!mbar_test(bar, parity) && now_ns() - t0 < kWaitNs) {
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
    d |= (uint64_t)1u << 16;                           // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1u << 46;                           // descriptor version for tcgen05
    d |= (uint64_t)2u << 61;                           // 128-byte swizzle
    return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Exact split of two FP32 values into packed BF16x2 hi / mid / lo terms.
__device__ __forceinline__ void split3(float a, float b, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
    const float ha = __uint_as_float(hi << 16), hb = __uint_as_float(hi & 0xFFFF0000u);
    const float ra = a - ha, rb = b - hb;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(mid) : "f"(rb), "f"(ra));
    const float ma = __uint_as_float(mid << 16), mb = __uint_as_float(mid & 0xFFFF0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(rb - mb), "f"(ra - ma));
}

struct TcParams {
    const float* A;
    int64_t lda, M, K;
    float* C;
    int64_t ldc;
    int S;            // valid output columns
    int N;            // MMA N (>= 16, multiple of 16)
    int astages;      // FP32 half-chunk ring depth
    int64_t tiles;
    int64_t kchunks;
    int* err;
};

__global__ void __launch_bounds__(kThreads, 1) right_tc_kernel(const __grid_constant__ CUtensorMap amap,
                                                               const __grid_constant__ CUtensorMap xmap,
                                                               const TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t a_full[4], a_empty[4];
    __shared__ __align__(8) uint64_t full_a[kSplitStages], full_b[kSplitStages], empty[kSplitStages];
    __shared__ __align__(8) uint64_t accf[2], acce[2], done_bar;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NA = p.astages;
    const uint32_t b_bytes = (uint32_t)p.N * kBK * 2;
    const uint32_t stage_bytes = 3 * kTermBytes + ((b_bytes + 1023u) & ~1023u);
    unsigned char* abuf = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sbuf = abuf + (size_t)NA * kHalfBytes;

    if (tid == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(&a_full[i], 1);
            mbar_init(&a_empty[i], kConvWarps * 32);
        }
        for (int i = 0; i < kSplitStages; ++i) {
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
    const uint32_t tmem_cols = (uint32_t)std::max(32, 1 << (32 - __clz(2 * p.N - 1)));
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s_tmem;

    // chunk sequence of this CTA: (tile, kc) for tile = blockIdx.x + i*gridDim.x
    const int64_t my_tiles = p.tiles > blockIdx.x ? (p.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total_chunks = my_tiles * p.kchunks;

    if (warp < kConvWarps) {
        // ---------------- converters: FP32 half chunks -> three BF16 tiles
        for (int64_t g = 0; g < total_chunks; ++g) {
            const int s = (int)(g % kSplitStages);
            if (!mbar_wait(&empty[s], (uint32_t)((g / kSplitStages) & 1) ^ 1u, &s_abort, p.err)) break;
            unsigned char* st = sbuf + (size_t)s * stage_bytes;
            bool ok = true;
            for (int h = 0; h < 2; ++h) {
                const int64_t hg = 2 * g + h;
                const int as = (int)(hg % NA);
                if (!mbar_wait(&a_full[as], (uint32_t)((hg / NA) & 1), &s_abort, p.err)) {
                    ok = false;
                    break;
                }
                const unsigned char* src = abuf + (size_t)as * kHalfBytes;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // rows {0,1,4,5} or {2,3,6,7} of an 8-row atom per instruction: the
                    // swizzled 8-byte stores of the four rows fall in two bank halves
                    const int gg = warp + 8 * j;
                    const int sel = lane >> 3, c4 = lane & 7;
                    const int roff = (sel & 1) * 4 + (sel >> 1);
                    const int r = 8 * (gg >> 1) + 2 * (gg & 1) + roff;
                    const float4 v = *reinterpret_cast<const float4*>(src + r * 128 + ((c4 ^ (r & 7)) << 4));
                    const int chunk16 = 4 * h + (c4 >> 1);
                    const uint32_t off = (uint32_t)r * 128u + ((uint32_t)(chunk16 ^ (r & 7)) << 4) +
                                         (uint32_t)(c4 & 1) * 8u;
                    uint32_t h0, m0, l0, h1, m1, l1;
                    split3(v.x, v.y, h0, m0, l0);
                    split3(v.z, v.w, h1, m1, l1);
                    *reinterpret_cast<uint2*>(st + off) = make_uint2(h0, h1);
                    *reinterpret_cast<uint2*>(st + kTermBytes + off) = make_uint2(m0, m1);
                    *reinterpret_cast<uint2*>(st + 2 * kTermBytes + off) = make_uint2(l0, l1);
                }
                mbar_arrive(&a_empty[as]);
            }
            if (!ok) break;
            fence_proxy_async();
            mbar_arrive(&full_a[s]);
        }
    } else if (warp == kAProdWarp) {
        // ---------------- TMA producer of A half chunks
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t hg = 0; hg < 2 * total_chunks; ++hg) {
                const int as = (int)(hg % NA);
                if (!mbar_wait(&a_empty[as], (uint32_t)((hg / NA) & 1) ^ 1u, &s_abort, p.err)) break;
                const int64_t g = hg >> 1;
                const int64_t tile = blockIdx.x + (g / p.kchunks) * gridDim.x;
                const int64_t kc = g % p.kchunks;
                mbar_arrive_expect_tx(&a_full[as], kHalfBytes);
                tma_load_2d(abuf + (size_t)as * kHalfBytes, &amap, (int)(kc * kBK + 32 * (hg & 1)),
                            (int)(tile * kBM), &a_full[as]);
                ++issued;
            }
            for (int64_t hg = std::max<int64_t>(0, issued - NA); hg < issued; ++hg)
                mbar_drain(&a_full[hg % NA], (uint32_t)((hg / NA) & 1));
        }
    } else if (warp == kBProdWarp) {
        // ---------------- TMA producer of X^T chunks
        if (lane == 0) {
            int64_t issued = 0;
            for (int64_t g = 0; g < total_chunks; ++g) {
                const int s = (int)(g % kSplitStages);
                if (!mbar_wait(&empty[s], (uint32_t)((g / kSplitStages) & 1) ^ 1u, &s_abort, p.err)) break;
                mbar_arrive_expect_tx(&full_b[s], b_bytes);
                tma_load_2d(sbuf + (size_t)s * stage_bytes + 3 * kTermBytes, &xmap, (int)((g % p.kchunks) * kBK), 0,
                            &full_b[s]);
                ++issued;
            }
            for (int64_t g = std::max<int64_t>(0, issued - kSplitStages); g < issued; ++g)
                mbar_drain(&full_b[g % kSplitStages], (uint32_t)((g / kSplitStages) & 1));
        }
    } else if (warp == kMmaWarp) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(p.N);
            int64_t g = 0;
            bool ok = true;
            for (int64_t it = 0; it < my_tiles && ok; ++it) {
                const int a = (int)(it & 1);
                if (!mbar_wait(&acce[a], (uint32_t)(((it >> 1) & 1) ^ 1), &s_abort, p.err)) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(a * p.N);
                for (int64_t kc = 0; kc < p.kchunks; ++kc, ++g) {
                    const int s = (int)(g % kSplitStages);
                    const uint32_t ph = (uint32_t)((g / kSplitStages) & 1);
                    if (!mbar_wait(&full_a[s], ph, &s_abort, p.err) ||
                        !mbar_wait(&full_b[s], ph, &s_abort, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t st = smem_u32(sbuf + (size_t)s * stage_bytes);
#pragma unroll
                    for (int kk = 0; kk < kBK / 16; ++kk) {
                        const uint64_t bdesc = sw128_desc(st + 3 * kTermBytes + 32u * kk);
#pragma unroll
                        for (int term = 0; term < 3; ++term) {
                            const uint64_t adesc = sw128_desc(st + term * kTermBytes + 32u * kk);
                            mma_bf16(d_tmem, adesc, bdesc, idesc, (kc | kk | term) ? 1u : 0u);
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
        // ---------------- epilogue warps 8..11: TMEM lanes 32*(warp%4) ..
        const int q = warp & 3;
        for (int64_t it = 0; it < my_tiles; ++it) {
            const int a = (int)(it & 1);
            if (!mbar_wait(&accf[a], (uint32_t)((it >> 1) & 1), &s_abort, p.err)) break;
            tc_fence_after();
            const int64_t tile = blockIdx.x + it * gridDim.x;
            const int64_t row = tile * kBM + q * 32 + lane;
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * p.N);
            for (int c = 0; c < p.N; c += 16) {
                float v[16];
                tmem_ld16(taddr + (uint32_t)c, v);
                if (row < p.M) {
                    float* dst = p.C + row * p.ldc + c;
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        if (c + j < p.S) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tmem_cols)
                     : "memory");
    }
}

// ---- host side --------------------------------------------------------------
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(ptr);
    }
    return fn;
}

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
                            int64_t ldc, int* err_flag, cudaStream_t st) {
    if (s <= 0 || A.rows <= 0) return cudaSuccess;
    if (s > 256 || s % 8 != 0) return cudaErrorInvalidValue;
    const int N = tc_mma_n(s);
    EncodeTiled enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t gdim[2] = {(cuuint64_t)ldt, (cuuint64_t)N};
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
    p.astages = N <= 128 ? 4 : 3;
    p.tiles = (A.rows + kBM - 1) / kBM;
    p.kchunks = (A.cols + kBK - 1) / kBK;
    p.err = err_flag;
    const uint32_t b_bytes = (uint32_t)N * kBK * 2;
    const size_t stage_bytes = 3 * kTermBytes + ((b_bytes + 1023u) & ~1023u);
    const size_t smem = (size_t)kHalfBytes * p.astages + stage_bytes * kSplitStages + 1024;
    cudaError_t e = cudaFuncSetAttribute(right_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (!g_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    }
    const int64_t grid = std::min<int64_t>(p.tiles, g_sms);
    right_tc_kernel<<<(unsigned)grid, kThreads, smem, st>>>(amap, map, p);
    return cudaGetLastError();
}

}  // namespace re
