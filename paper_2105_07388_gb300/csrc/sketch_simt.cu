// FP32 CUDA-core kernels of the two-sided sketch Y*A*X (Algorithm 1 steps 3 and 6).
//
//  * right_simt: A*X (step 3) for a Gaussian X held as an FP32 n x s buffer.
//    A is streamed once per column tile; 128-row x BN-column CTA tiles, K steps
//    of 32, A staged through registers into a k-major shared tile so that each
//    thread runs an 8 x TN outer product per k.  FP64 input is rounded to FP32
//    as it is loaded.  Transposed orientation (m < n) reads A by columns.
//  * left_sketch: Y*(A X) (step 6) as split-K partial products over the long
//    dimension m, with Y generated on the fly (Gaussian from the counter-based
//    generator, or SRTT entries d_i (-1)^popcount(pi(q) & i)), reduced in FP64
//    in a fixed order.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 32;
constexpr int kThreads = 256;

template <int BN>
struct SimtShape;
template <> struct SimtShape<128> { static constexpr int TN = 8; };
template <> struct SimtShape<64> { static constexpr int TN = 4; };
template <> struct SimtShape<32> { static constexpr int TN = 2; };
template <> struct SimtShape<16> { static constexpr int TN = 1; };
template <> struct SimtShape<8> { static constexpr int TN = 1; };

template <typename TA>
__device__ __forceinline__ float ld_as_f32(const TA* p) {
    return (float)__ldg(p);
}

// Loads of one BM x 32 A tile into registers (BM/8 values per thread).
// Non-transposed: thread t holds row (t % BM), k range [(t / BM) * BM/8, + BM/8).
// Transposed (oriented (r, c) = A[c * lda + r]): thread t holds k = t / 8 and
// rows [(t % 8) * BM/8, + BM/8).
template <typename TA, bool TRANS, int BM>
struct ATile {
    static constexpr int PER = BM / 8;
    float v[PER];

    __device__ __forceinline__ void load(const TA* __restrict__ A, int64_t lda, int64_t M,
                                         int64_t N, int64_t m0, int64_t k0, bool vec) {
        const int t = threadIdx.x;
        if (!TRANS) {
            const int64_t r = m0 + (t % BM);
            const int64_t kb = k0 + PER * (t / BM);
            if constexpr (sizeof(TA) == 4) {
                if (vec && r < M && kb + PER <= N) {
                    const float4* p = reinterpret_cast<const float4*>(A + r * lda + kb);
#pragma unroll
                    for (int q = 0; q < PER / 4; ++q) {
                        const float4 w = __ldg(p + q);
                        v[4 * q + 0] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
                    }
                    return;
                }
            }
#pragma unroll
            for (int q = 0; q < PER; ++q)
                v[q] = (r < M && kb + q < N) ? ld_as_f32(A + r * lda + kb + q) : 0.0f;
        } else {
            const int64_t c = k0 + (t >> 3);
            const int64_t rb = m0 + PER * (t & 7);
            if constexpr (sizeof(TA) == 4) {
                if (vec && c < N && rb + PER <= M) {
                    const float4* p = reinterpret_cast<const float4*>(A + c * lda + rb);
#pragma unroll
                    for (int q = 0; q < PER / 4; ++q) {
                        const float4 w = __ldg(p + q);
                        v[4 * q + 0] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
                    }
                    return;
                }
            }
#pragma unroll
            for (int q = 0; q < PER; ++q)
                v[q] = (c < N && rb + q < M) ? ld_as_f32(A + c * lda + rb + q) : 0.0f;
        }
    }

    // shared tile layout: As[k][m] with row pitch BM + 4
    __device__ __forceinline__ void store(float* As) const {
        const int t = threadIdx.x;
        if (!TRANS) {
            const int r = t % BM;
            const int kb = PER * (t / BM);
#pragma unroll
            for (int q = 0; q < PER; ++q) As[(kb + q) * (BM + 4) + r] = v[q];
        } else {
            const int c = t >> 3;
            const int rb = PER * (t & 7);
            float4* p = reinterpret_cast<float4*>(As + c * (BM + 4) + rb);
#pragma unroll
            for (int q = 0; q < PER / 4; ++q) p[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    }
};

template <int BN>
struct XTile {
    static constexpr int PER = BN / 8;   // floats per thread (32 x BN tile, 256 threads)
    float v[PER];

    __device__ __forceinline__ void load(const float* __restrict__ X, int64_t ldx, int64_t N,
                                         int64_t k0, int n0, int ncols) {
        const int t = threadIdx.x;
        const int64_t k = k0 + (t >> 3);
        const int c = n0 + (t & 7) * PER;
#pragma unroll
        for (int q = 0; q < PER; ++q) v[q] = (k < N && c + q < ncols) ? __ldg(X + k * ldx + c + q) : 0.0f;
    }

    __device__ __forceinline__ void store(float* Bs) const {
        const int t = threadIdx.x;
        const int k = t >> 3;
        const int c = (t & 7) * PER;
#pragma unroll
        for (int q = 0; q < PER; ++q) Bs[k * BN + c + q] = v[q];
    }
};

// One BM x BN output tile of A*X (FP32 FMA): rows m0.., columns n0.. of C.
// smem: 2 x 32 x (BM+4) floats for A, then 2 x 32 x BN floats for X.
template <int BN, bool TRANS, typename TA, int BM>
__device__ __forceinline__ void simt_tile(const TA* __restrict__ A, int64_t lda, int64_t M, int64_t N,
                                          const float* __restrict__ X, int64_t ldx,
                                          float* __restrict__ C, int64_t ldc, int64_t m0, int n0,
                                          bool vec, float* smem, int ncols) {
    using S = SimtShape<BN>;
    constexpr int TN = S::TN;
    constexpr int TX = BN / TN;
    constexpr int TY = kThreads / TX;
    constexpr int TM = BM / TY;
    static_assert(TM % 4 == 0 || TM == 2, "row fragment");
    float* As = smem;                                // 2 x kBK x (BM+4)
    float* Bs = As + 2 * kBK * (BM + 4);             // 2 x kBK x BN
    const int tx = threadIdx.x % TX;
    const int ty = threadIdx.x / TX;

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0f;

    ATile<TA, TRANS, BM> at;
    XTile<BN> xt;
    const int64_t KT = (N + kBK - 1) / kBK;
    at.load(A, lda, M, N, m0, 0, vec);
    xt.load(X, ldx, N, 0, n0, ncols);
    at.store(As);
    xt.store(Bs);
    __syncthreads();

    for (int64_t kt = 0; kt < KT; ++kt) {
        const int buf = (int)(kt & 1);
        const bool more = kt + 1 < KT;
        if (more) {
            at.load(A, lda, M, N, m0, (kt + 1) * kBK, vec);
            xt.load(X, ldx, N, (kt + 1) * kBK, n0, ncols);
        }
        const float* as = As + buf * kBK * (BM + 4);
        const float* bs = Bs + buf * kBK * BN;
#pragma unroll 8
        for (int k = 0; k < kBK; ++k) {
            float a[TM], b[TN];
            const float* ap = as + k * (BM + 4) + ty * TM;
            if constexpr (TM >= 4) {
#pragma unroll
                for (int i = 0; i < TM; i += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(ap + i);
                    a[i] = w.x; a[i + 1] = w.y; a[i + 2] = w.z; a[i + 3] = w.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = ap[i];
            }
            const float* bp = bs + k * BN + tx * TN;
            if constexpr (TN >= 4) {
#pragma unroll
                for (int j = 0; j < TN; j += 4) {
                    const float4 w = *reinterpret_cast<const float4*>(bp + j);
                    b[j] = w.x; b[j + 1] = w.y; b[j + 2] = w.z; b[j + 3] = w.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = bp[j];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            at.store(As + (buf ^ 1) * kBK * (BM + 4));
            xt.store(Bs + (buf ^ 1) * kBK * BN);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int64_t r = m0 + ty * TM + i;
        if (r >= M) continue;
        float* cp = C + r * ldc + n0 + tx * TN;
#pragma unroll
        for (int j = 0; j < TN; ++j)
            if (n0 + tx * TN + j < ncols) cp[j] = acc[i][j];
    }
}

template <int BN, bool TRANS, typename TA>
__global__ void __launch_bounds__(kThreads) right_simt_kernel(const TA* __restrict__ A, int64_t lda,
                                                              int64_t M, int64_t N,
                                                              const float* __restrict__ X,
                                                              int64_t ldx, float* __restrict__ C,
                                                              int64_t ldc, int vec, int ncols) {
    extern __shared__ float4 smem_raw[];
    simt_tile<BN, TRANS, TA, kBM>(A, lda, M, N, X, ldx, C, ldc, (int64_t)blockIdx.y * kBM,
                                  (int)blockIdx.x * BN, vec != 0, reinterpret_cast<float*>(smem_raw), ncols);
}

// Batched: one CTA per (block, BM-row tile) work item.
__device__ __forceinline__ int find_block(const int64_t* prefix, int count, int64_t item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int BN, int BM>
__global__ void __launch_bounds__(kThreads) right_simt_batched_kernel(
    const BatchDesc* __restrict__ d, int count, const int64_t* __restrict__ tile_prefix,
    const int* __restrict__ active, const float* __restrict__ Xpool, int s,
    float* __restrict__ AXpool, int64_t ldax, int col0) {
    extern __shared__ float4 smem_raw[];
    const int64_t item = blockIdx.x;
    const int b = find_block(tile_prefix, count, item);
    if (!active[b]) return;
    const BatchDesc D = d[b];
    const int64_t m0 = (item - tile_prefix[b]) * BM;
    const bool vec = ((reinterpret_cast<uintptr_t>(D.A) & 15) == 0) && ((D.ld & 3) == 0);
    const float* X = Xpool + D.x_off;
    float* C = AXpool + D.ax_off + col0;
    float* sm = reinterpret_cast<float*>(smem_raw);
    if (D.trans)
        simt_tile<BN, true, float, BM>(D.A, D.ld, D.rows, D.cols, X, s, C, ldax, m0, 0, vec, sm, s);
    else
        simt_tile<BN, false, float, BM>(D.A, D.ld, D.rows, D.cols, X, s, C, ldax, m0, 0, vec, sm, s);
}

template <int BN, int BM>
cudaError_t launch_batched_t(const BatchDesc* d, int count, const int64_t* tile_prefix, int64_t items,
                             const int* active, const float* Xpool, int s, float* AXpool, int64_t ldax,
                             int col0, cudaStream_t st) {
    const size_t smem = sizeof(float) * (2 * kBK * (BM + 4) + 2 * kBK * BN);
    auto kern = right_simt_batched_kernel<BN, BM>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)items, kThreads, smem, st>>>(d, count, tile_prefix, active, Xpool, s, AXpool, ldax, col0);
    return cudaGetLastError();
}

template <int BM>
cudaError_t dispatch_batched(const BatchDesc* d, int count, const int64_t* tile_prefix, int64_t items,
                             const int* active, const float* Xpool, int s, float* AXpool, int64_t ldax,
                             int col0, cudaStream_t st) {
    switch (s) {
        case 8: return launch_batched_t<8, BM>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
        case 16: return launch_batched_t<16, BM>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
        case 32: return launch_batched_t<32, BM>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
        case 64: return launch_batched_t<64, BM>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
        case 128: return launch_batched_t<128, BM>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int BN, bool TRANS, typename TA>
cudaError_t launch_right_simt_t(const MatView& A, const float* X, int64_t ldx, int s, float* C,
                                int64_t ldc, cudaStream_t st) {
    const size_t smem = sizeof(float) * (2 * kBK * (kBM + 4) + 2 * kBK * BN);
    auto kern = right_simt_kernel<BN, TRANS, TA>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    const int vec = ((reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0 && (A.ld & 3) == 0) ? 1 : 0;
    dim3 grid((unsigned)((s + BN - 1) / BN), (unsigned)((A.rows + kBM - 1) / kBM));
    kern<<<grid, kThreads, smem, st>>>(static_cast<const TA*>(A.ptr), A.ld, A.rows, A.cols, X, ldx,
                                        C, ldc, vec, s);
    return cudaGetLastError();
}

template <int BN>
cudaError_t dispatch_right(const MatView& A, const float* X, int64_t ldx, int s, float* C,
                           int64_t ldc, cudaStream_t st) {
    if (A.dtype == RE_F32) {
        return A.trans ? launch_right_simt_t<BN, true, float>(A, X, ldx, s, C, ldc, st)
                       : launch_right_simt_t<BN, false, float>(A, X, ldx, s, C, ldc, st);
    }
    return A.trans ? launch_right_simt_t<BN, true, double>(A, X, ldx, s, C, ldc, st)
                   : launch_right_simt_t<BN, false, double>(A, X, ldx, s, C, ldc, st);
}

// ---------------------------------------------------------------------------
// Left sketch: part[split][r][c] = sum over the split's rows i of
// Y[row0+r][i] AX[i][col0+c], Y Gaussian (normals of stream GY) or, with DCT,
// the SRCT rows of Yd generated from the cosine table.
constexpr int kLR = 64;     // rows of Y per tile
constexpr int kLK = 32;     // i per k step

// Entry (q, i) of the unscaled SRCT left embedding (see DctRows): the phase
// (2i+1) k is reduced modulo 4N in integers, then folded onto [0, N] by the
// symmetries cos(2 pi - x) = cos x and cos(pi - x) = -cos x.
__device__ __forceinline__ float dct_entry(const DctRows& Y, int q, int64_t i, float d) {
    const int k = __ldg(Y.krow + q);
    if (k == 0) return d;
    const unsigned long long N = 1ull << Y.nbits;
    unsigned long long ph = ((2ull * (unsigned long long)i + 1ull) * (unsigned long long)k) & (4ull * N - 1ull);
    if (ph > 2ull * N) ph = 4ull * N - ph;
    const float c = ph <= N ? __ldg(Y.ctab + ph) : -__ldg(Y.ctab + (2ull * N - ph));
    return 1.41421356237309515f * c * d;
}

template <int LC, bool DCT>
__global__ void __launch_bounds__(256) left_kernel(uint64_t seed, const float* __restrict__ AX,
                                                   int64_t ldax, int64_t M, int row0, int R,
                                                   int col0, int S, int64_t chunk,
                                                   float* __restrict__ part, const DctRows Yd) {
    constexpr int TC = LC / 16;           // columns per thread
    __shared__ __align__(16) float Ys[kLK][kLR];
    __shared__ __align__(16) float Xs[kLK][LC];
    const int ct = blockIdx.x, rt = blockIdx.y, split = blockIdx.z;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;           // 16 x 16 threads, 4 rows x TC cols each
    const int64_t i_begin = (int64_t)split * chunk;
    const int64_t i_end = min(M, i_begin + chunk);
    const int qbase = row0 + rt * kLR;                // first Y row of this tile (multiple of 8)

    float acc[4][TC];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < TC; ++b) acc[a][b] = 0.0f;

    for (int64_t i0 = i_begin; i0 < i_end; i0 += kLK) {
        // ---- Y tile: Ys[k][r] = Y[qbase + r][i0 + k]
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = tid & 31;
            const int g = (tid >> 5) + 8 * h;            // 16 groups of 4 rows
            const int64_t i = i0 + k;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (DCT) {
                if (i < i_end) {
                    const float d = ((__ldg(Yd.dbits + (i >> 5)) >> (i & 31)) & 1u) ? -1.f : 1.f;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int q = qbase + 4 * g + a;
                        if (q - row0 < R) z[a] = dct_entry(Yd, q, i, d);
                    }
                }
            } else {
                if (i < i_end && qbase + 4 * g - row0 < R)
                    normals4((uint32_t)i, (uint32_t)((qbase >> 2) + g), kStreamGY, seed, z);
            }
            *reinterpret_cast<float4*>(&Ys[k][4 * g]) = make_float4(z[0], z[1], z[2], z[3]);
        }
        // ---- AX tile: Xs[k][c] = AX[i0 + k][col0 + ct*LC + c]
        {
            constexpr int PER = LC * kLK / 256;
            const int k = tid / (LC / PER);
            const int cb = (tid % (LC / PER)) * PER;
            const int64_t i = i0 + k;
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int c = ct * LC + cb + q;
                Xs[k][cb + q] = (i < i_end && c < S) ? __ldg(AX + i * ldax + col0 + c) : 0.0f;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < kLK; ++k) {
            const float4 yv = *reinterpret_cast<const float4*>(&Ys[k][ty * 4]);
            const float y[4] = {yv.x, yv.y, yv.z, yv.w};
            float x[TC];
#pragma unroll
            for (int b = 0; b < TC; b += 4) {
                const float4 w = *reinterpret_cast<const float4*>(&Xs[k][tx * TC + b]);
                x[b] = w.x; x[b + 1] = w.y; x[b + 2] = w.z; x[b + 3] = w.w;
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < TC; ++b) acc[a][b] = fmaf(y[a], x[b], acc[a][b]);
        }
        __syncthreads();
    }
    // part layout: [split][R][S]
    float* out = part + (int64_t)split * R * S;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = rt * kLR + ty * 4 + a;
        if (r >= R) continue;
#pragma unroll
        for (int b = 0; b < TC; ++b) {
            const int c = ct * LC + tx * TC + b;
            if (c < S) out[(int64_t)r * S + c] = acc[a][b];
        }
    }
}

// core block = sum of the split-K partials, in FP64 and in a fixed order: a CTA
// owns 32 consecutive outputs (one per lane, so every load is a 128-byte line),
// warp w sums splits w, w+8, w+16, ..., and the 8 warp sums are added in warp
// order (the result does not depend on scheduling).
// Sum of the split-K partials of each core entry, in a fixed order (lanes over
// entries, warps over splits, then warp 0 combines the 8 warp sums).  Each warp
// accumulates in FP32 with an error-free TwoSum correction (s + c carries the
// sum to about u^2 relative, as good as an FP64 accumulation for these term
// counts) because FP64 adds issue at 1/64 of the FP32 rate on this part.
__global__ void __launch_bounds__(256) left_reduce_kernel(const float* __restrict__ part, int splits, int R,
                                                          int S, int row0, int col0, double* __restrict__ core,
                                                          int64_t ld_core) {
    __shared__ float s_hi[8][32], s_lo[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t total = (int64_t)R * S;
    const int64_t idx = (int64_t)blockIdx.x * 32 + lane;
    float sum = 0.f, comp = 0.f;
    if (idx < total)
        for (int p = w; p < splits; p += 8) {
            const float x = part[(int64_t)p * total + idx];
            const float t = sum + x;                       // TwoSum(sum, x)
            const float bp = t - sum;
            comp += (sum - (t - bp)) + (x - bp);
            sum = t;
        }
    s_hi[w][lane] = sum;
    s_lo[w][lane] = comp;
    __syncthreads();
    if (w == 0 && idx < total) {
        double t = (double)s_hi[0][lane] + (double)s_lo[0][lane];
#pragma unroll
        for (int u = 1; u < 8; ++u) t += (double)s_hi[u][lane] + (double)s_lo[u][lane];
        const int r = (int)(idx / S), c = (int)(idx % S);
        core[(int64_t)(row0 + r) * ld_core + col0 + c] = t;
    }
}

int left_splits(int64_t M, int R, int S, int64_t* chunk_out) {
    const int tiles = ((R + kLR - 1) / kLR) * ((S + 63) / 64);
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>((M + 1023) / 1024, (4 * 152 + tiles - 1) / tiles));
    int64_t chunk = (M + splits - 1) / splits;
    chunk = (chunk + kLK - 1) / kLK * kLK;
    splits = (int)((M + chunk - 1) / chunk);
    *chunk_out = chunk;
    return splits;
}

}  // namespace

cudaError_t launch_right_simt(const MatView& A, const float* X, int64_t ldx, int s, float* C,
                              int64_t ldc, cudaStream_t st) {
    if (s <= 0 || A.rows <= 0) return cudaSuccess;
    if ((A.rows + kBM - 1) / kBM > 65535) return cudaErrorInvalidConfiguration;
    // one launch for any width: 128-wide column tiles (the last one masked) from
    // 128 columns up, otherwise the narrowest tile that covers all columns; the
    // column tiles of a row block run back to back, so A streams from HBM once
    if (s >= 128 || s > 64) return dispatch_right<128>(A, X, ldx, s, C, ldc, st);
    if (s > 32) return dispatch_right<64>(A, X, ldx, s, C, ldc, st);
    if (s > 16) return dispatch_right<32>(A, X, ldx, s, C, ldc, st);
    if (s > 8) return dispatch_right<16>(A, X, ldx, s, C, ldc, st);
    return dispatch_right<8>(A, X, ldx, s, C, ldc, st);
}

cudaError_t launch_right_simt_batched(const BatchDesc* d, int count, const int64_t* tile_prefix,
                                      int64_t items, const int* active, const float* Xpool, int s,
                                      float* AXpool, int64_t ldax, int col0, int bm, cudaStream_t st) {
    if (items <= 0) return cudaSuccess;
    if (bm == 64) return dispatch_batched<64>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
    return dispatch_batched<128>(d, count, tile_prefix, items, active, Xpool, s, AXpool, ldax, col0, st);
}

size_t left_part_floats(int64_t M, int R, int S) {
    int64_t chunk;
    const int splits = left_splits(M, R, S, &chunk);
    return (size_t)splits * R * S;
}

cudaError_t launch_left(uint64_t seed, const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0, int S,
                        float* part, size_t part_cap, double* core, int64_t ld_core, cudaStream_t st,
                        int* err_flag) {
    if (R <= 0 || S <= 0) return cudaSuccess;
    if (err_flag && left_tc_supported(AX, ldax, M, row0, R, col0, S) &&
        left_tc_part_floats(M, R, S) <= part_cap) {
        int tsplits = 0;
        cudaError_t e = launch_left_tc_partials(seed, AX, ldax, M, row0, R, col0, S, part, part_cap, err_flag,
                                                &tsplits, st);
        if (e != cudaSuccess) return e;
        const int64_t total = (int64_t)R * S;
        left_reduce_kernel<<<(unsigned)((total + 31) / 32), 256, 0, st>>>(part, tsplits, R, S, row0, col0,
                                                                                 core, ld_core);
        return cudaGetLastError();
    }
    int64_t chunk;
    const int splits = left_splits(M, R, S, &chunk);
    if ((size_t)splits * R * S > part_cap) return cudaErrorInvalidValue;
    const bool wide = S >= 128;
    dim3 grid((unsigned)((S + (wide ? 127 : 63)) / (wide ? 128 : 64)), (unsigned)((R + kLR - 1) / kLR),
              (unsigned)splits);
    const DctRows none{nullptr, nullptr, nullptr, 0};
    if (wide)
        left_kernel<128, false><<<grid, 256, 0, st>>>(seed, AX, ldax, M, row0, R, col0, S, chunk, part, none);
    else
        left_kernel<64, false><<<grid, 256, 0, st>>>(seed, AX, ldax, M, row0, R, col0, S, chunk, part, none);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)R * S;
    left_reduce_kernel<<<(unsigned)((total + 31) / 32), 256, 0, st>>>(part, splits, R, S, row0, col0,
                                                                             core, ld_core);
    return cudaGetLastError();
}

cudaError_t launch_left_dct(const DctRows& Y, const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0,
                            int S, float* part, size_t part_cap, double* core, int64_t ld_core, cudaStream_t st,
                            int* err_flag) {
    if (R <= 0 || S <= 0) return cudaSuccess;
    if (err_flag && left_tc_supported(AX, ldax, M, row0, R, col0, S) &&
        left_tc_part_floats(M, R, S, true) <= part_cap) {
        int tsplits = 0;
        cudaError_t e = launch_left_tc_partials(0, AX, ldax, M, row0, R, col0, S, part, part_cap, err_flag, &tsplits,
                                                st, &Y);
        if (e != cudaSuccess) return e;
        const int64_t total = (int64_t)R * S;
        left_reduce_kernel<<<(unsigned)((total + 31) / 32), 256, 0, st>>>(part, tsplits, R, S, row0, col0,
                                                                                 core, ld_core);
        return cudaGetLastError();
    }
    int64_t chunk;
    const int splits = left_splits(M, R, S, &chunk);
    if ((size_t)splits * R * S > part_cap) return cudaErrorInvalidValue;
    const bool wide = S >= 128;
    dim3 grid((unsigned)((S + (wide ? 127 : 63)) / (wide ? 128 : 64)), (unsigned)((R + kLR - 1) / kLR),
              (unsigned)splits);
    if (wide)
        left_kernel<128, true><<<grid, 256, 0, st>>>(0, AX, ldax, M, row0, R, col0, S, chunk, part, Y);
    else
        left_kernel<64, true><<<grid, 256, 0, st>>>(0, AX, ldax, M, row0, R, col0, S, chunk, part, Y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)R * S;
    left_reduce_kernel<<<(unsigned)((total + 31) / 32), 256, 0, st>>>(part, splits, R, S, row0, col0, core, ld_core);
    return cudaGetLastError();
}

}  // namespace re
