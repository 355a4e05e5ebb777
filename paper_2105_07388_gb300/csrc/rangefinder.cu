// Algorithm 3 (Sec. 5.1, rank estimation combined with the randomized
// rangefinder) after the sketch: the rank selection of step 5 and the thin QR of
// step 7 and product of step 8 for the first k = r + p columns of A X.
//
// Step 5 (`select_rank_kernel`): the smallest r in [0, min(r1, n)] with
//   (1 + r/(p-1))^{1/2} (sum_{j>r} sigma^_j^2)^{1/2} <= eps ||A||,
// sigma^_j = sigma^_{r1} for r1 < j <= n (step 4), values beyond the n-th zero,
// in FP64 on one thread.
//
// Step 7 by sketch-to-precondition (the randomized approximate orthogonalization
// of Sec. 4): the core Y (A X_k) is a sketch of A X_k, so with R_s its triangular
// factor, W = (A X_k) R_s^{-1} is well conditioned whatever A X_k's condition
// number (about 1e7 when the p extra columns sit at the FP32 noise floor); two
// Cholesky-QR passes on W then give Q with orthonormal columns, and the leading
// columns of Q span the same nested subspaces as those of A X_k.  R_s comes from
// the FP64 Cholesky factor of the core's Gram matrix (k x k; the core is FP64, so
// its Gram keeps the squared condition number, 1e14, inside FP64).  Small
// factorizations (Cholesky, triangular inverse; k <= 1024) run in one CTA, in
// FP64 for R_s and in FP32 for the two passes on the well-conditioned W.
//
// Products (all kernels of this file, no library GEMM):
//   the core's Gram    FP64, 32 x 32 output tiles (`gram64_kernel`);
//   W = (A X_k) L^{-T} FP32 CUDA-core tiles of 128 x 128 (`sgemm_kernel`);
//   V^T V              the same tiles, split over the rows of V, the partial
//                      Gram matrices summed in FP64 in a fixed order;
//   B = Q^T A          the same tiles (A read once per 128 columns of Q), split
//                      over the rows of A when the output has few tiles.
#include <climits>
#include <cmath>
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {


// Steps 4-5 of Algorithm 3 (one warp): lane 0 accumulates the tail sums T(r) from
// the end, in the order of the sequential definition; the lanes then test the
// criterion for r = lane, lane + 32, ... (two square roots and a division each,
// the costly part in FP64) and a warp minimum keeps the smallest r that meets it.
constexpr int kSelMax = 1024;       // trusted values held in shared memory (r1 <= 465 at s = 512)

__global__ void select_rank_kernel(const double* __restrict__ sig, int r1, int64_t n, double eps, double norm_a,
                                   int p, int s, QbSelect* __restrict__ out) {
    __shared__ double Ts[kSelMax + 1];
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const double ref = norm_a > 0.0 ? norm_a : (r1 > 0 ? sig[0] : 0.0);
    // A has only n singular values: a sketch wider than n trusts at most n of them
    int re = (int)(n < (int64_t)r1 ? n : (int64_t)r1);
    if (re > kSelMax) re = kSelMax;
    if (lane == 0) {
        const double last = re > 0 ? sig[re - 1] : 0.0;
        // T(r) = sum_{j>r} sigma^_j^2, accumulated from the tail: T(re) = (n - re) sigma^_{re}^2
        double T = (double)(n - re) * last * last;
        Ts[re] = T;
        for (int r = re - 1; r >= 0; --r) {
            T += sig[r] * sig[r];
            Ts[r] = T;
        }
    }
    __syncwarp();
    int best = INT_MAX;
    double best_bound = 0.0;
    for (int r = lane; r <= re; r += 32) {
        const double bound = sqrt(1.0 + (double)r / (p - 1.0)) * sqrt(Ts[r]);
        if (bound <= eps * ref && r < best) {
            best = r;
            best_bound = bound;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int b2 = __shfl_xor_sync(0xffffffffu, best, o);
        const double v2 = __shfl_xor_sync(0xffffffffu, best_bound, o);
        if (b2 < best) {
            best = b2;
            best_bound = v2;
        }
    }
    if (lane != 0) return;
    if (best == INT_MAX) best = -1;
    out->r = best;
    // k = min(r + p, n) columns factor A exactly once the sketch covers all n
    // singular values, so the criterion is met when those k columns are sketched
    const int64_t k = (int64_t)best + p < n ? (int64_t)best + p : n;
    out->met = (best >= 0 && k <= s) ? 1 : 0;
    out->bound = best_bound;
    out->norm_a = ref;
}

// ---- blocked FP64 Cholesky factorization and triangular inverse (k <= 1024)
// Both work on kp x kp row-major matrices, kp = the power of two >= k (at least
// kTB = 32), the k x k matrix padded with the identity (so the padding factors
// and inverts to the identity and never mixes with the leading block).
//
// Cholesky G = L L^T, right-looking by 32-column block steps J: every CTA of
// `blk_potrf_trsm_kernel` factors the diagonal block (J, J) (redundantly, in
// shared memory) and CTA c > 0 then solves the block (J + c, J) against it;
// `blk_syrk_kernel` subtracts L(I, J) L(K, J)^T from every trailing tile
// J < K <= I.  Deflation: a pivot d_j (the squared norm of what column j adds
// to the span of the earlier columns) not above rel * G_jj, or not above 1e-30
// of G's largest diagonal entry, marks column j as numerically dependent: its
// pivot becomes 1, the entries below it 0 (so nothing of it reaches the later
// columns), defl[j] = 1 and *floored is set; the inverse's row j is then
// written as zeros, and the orthonormalised column j comes out as zero.
//
// Inverse X = L^{-1} by recursive doubling: the 32 x 32 diagonal blocks are
// inverted by forward substitution, then for block size s = 32, 64, ...: with
// [[A, 0], [B, C]] a diagonal block of size 2s, its lower-left block of the
// inverse is -C^{-1} (B A^{-1}) -- two batched FP64 products per level.
constexpr int kTB = 32;

__global__ void blk_init_kernel(const double* __restrict__ G, int ldg, int k, int kp, double* __restrict__ Lp) {
    const int64_t total = (int64_t)kp * kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / kp), j = (int)(e % kp);
        double v = 0.0;
        if (i < k && j < k) v = j <= i ? G[(int64_t)i * ldg + j] : 0.0;
        else if (i == j) v = 1.0;
        Lp[e] = v;
    }
}

__global__ void blk_floor_kernel(const double* __restrict__ G, int ldg, int k, double* __restrict__ fl) {
    __shared__ double red[32];
    double mx = 0.0;
    for (int i = threadIdx.x; i < k; i += blockDim.x) mx = fmax(mx, G[(int64_t)i * ldg + i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        fl[0] = mx > 0.0 ? mx * 1e-30 : 1.0;   // an all-zero Gram matrix (A X_k = 0): every column deflates
    }
}

// 32 x 32 lower Cholesky factorization of D (shared, row pitch kTB + 1) by the
// 1024 threads of the block, thread (r, c) = (tid / 32, tid % 32).  thr[j] is
// column j's deflation threshold; dfl[j] (shared) receives its mark.
// The pivot's square root and the column's scaling come from one reciprocal square
// root: L_jj = d rsqrt(d) and L_rj = D_rj rsqrt(d), so each of the 32 steps waits
// for one long FP64 operation instead of a square root and then a division
// (FP64 instructions issue at a small fraction of the FP32 rate on this GPU).
__device__ void potrf32(double (*D)[kTB + 1], const double* thr, int* dfl) {
    __shared__ double s_rinv;
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    for (int j = 0; j < kTB; ++j) {
        if (r == j && c == j) {
            const double d = D[j][j];
            const bool dep = !(d > thr[j]);
            dfl[j] = dep ? 1 : 0;
            const double y = dep ? 1.0 : rsqrt(d);
            D[j][j] = dep ? 1.0 : d * y;
            s_rinv = y;
        }
        __syncthreads();
        if (c == j && r > j) D[r][j] = dfl[j] ? 0.0 : D[r][j] * s_rinv;
        __syncthreads();
        if (r > j && c > j && c <= r) D[r][c] -= D[r][j] * D[c][j];
        __syncthreads();
    }
}

// X (shared) = D^{-1} for the lower-triangular D: thread c of warp 0 owns column c.
// The diagonal's reciprocals are formed once, in parallel, so the substitution
// multiplies instead of dividing at each of its steps.
__device__ void trinv32(const double (*D)[kTB + 1], double (*X)[kTB + 1]) {
    __shared__ double rd[kTB];
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    X[r][c] = 0.0;
    if (threadIdx.x < kTB) rd[c] = 1.0 / D[c][c];
    __syncthreads();
    if (threadIdx.x < kTB) {
        X[c][c] = rd[c];
        for (int i = c + 1; i < kTB; ++i) {
            double acc = 0.0;
            for (int l = c; l < i; ++l) acc = fma(D[i][l], X[l][c], acc);
            X[i][c] = -acc * rd[i];
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(1024) blk_potrf_trsm_kernel(double* __restrict__ Lp, int kp, int J,
                                                              const double* __restrict__ G, int ldg, int k,
                                                              double rel, const double* __restrict__ fl,
                                                              int* __restrict__ defl, int* floored) {
    __shared__ double D[kTB][kTB + 1], Dinv[kTB][kTB + 1], P[kTB][kTB + 1];
    __shared__ double thr[kTB];
    __shared__ int dfl[kTB];
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    const int64_t j0 = (int64_t)J * kTB, i0 = j0 + (int64_t)blockIdx.x * kTB;
    D[r][c] = c <= r ? Lp[(j0 + r) * kp + j0 + c] : 0.0;
    if (r == 0) {
        const int64_t jj = j0 + c;
        // padding columns (identity) never deflate
        thr[c] = jj < k ? fmax(rel * G[jj * ldg + jj], fl[0]) : 0.0;
    }
    __syncthreads();
    potrf32(D, thr, dfl);
    if (blockIdx.x == 0) {
        Lp[(j0 + r) * kp + j0 + c] = c <= r ? D[r][c] : 0.0;
        if (r == 0) {
            defl[j0 + c] = dfl[c];
            if (dfl[c] && j0 + c < k && floored) *floored = 1;
        }
        return;
    }
    trinv32(D, Dinv);
    // L(I, J) = P D^{-T}: L[r][c] = sum_{l <= c} P[r][l] Dinv[c][l]; 0 in deflated columns
    P[r][c] = Lp[(i0 + r) * kp + j0 + c];
    __syncthreads();
    double acc = 0.0;
    for (int l = 0; l <= c; ++l) acc = fma(P[r][l], Dinv[c][l], acc);
    Lp[(i0 + r) * kp + j0 + c] = dfl[c] ? 0.0 : acc;
}

// Trailing update after step J: tile t of the lower triangle J < K <= I < nb
// (row-major order of the (I, K) pairs); 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256) blk_syrk_kernel(double* __restrict__ Lp, int kp, int J) {
    __shared__ double Ta[kTB][kTB + 1], Tb[kTB][kTB + 1];
    int t = (int)blockIdx.x, I = J + 1;
    while (t >= I - J) {                  // row I holds I - J tiles K = J+1 .. I
        t -= I - J;
        ++I;
    }
    const int K = J + 1 + t;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t j0 = (int64_t)J * kTB, ib = (int64_t)I * kTB, kb = (int64_t)K * kTB;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        Ta[ty + 8 * q][tx] = Lp[(ib + ty + 8 * q) * kp + j0 + tx];
        Tb[ty + 8 * q][tx] = Lp[(kb + ty + 8 * q) * kp + j0 + tx];
    }
    __syncthreads();
    // Lp[I][K] (r, c) -= sum_l Ta[r][l] Tb[c][l]
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int rr = ty + 8 * q;
        double acc = 0.0;
#pragma unroll 8
        for (int l = 0; l < kTB; ++l) acc = fma(Ta[rr][l], Tb[tx][l], acc);
        Lp[(ib + rr) * kp + kb + tx] -= acc;
    }
}

__global__ void __launch_bounds__(1024) blk_inv_diag_kernel(const double* __restrict__ Lp, int kp,
                                                            double* __restrict__ Xp) {
    __shared__ double D[kTB][kTB + 1], X[kTB][kTB + 1];
    const int r = threadIdx.x >> 5, c = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.x * kTB;
    D[r][c] = Lp[(j0 + r) * kp + j0 + c];
    __syncthreads();
    trinv32(D, X);
    // the whole block row of X: the diagonal block, zeros elsewhere (filled level by level)
    for (int64_t col = c; col < kp; col += kTB) {
        const bool diag = col >= j0 && col < j0 + kTB;
        Xp[(j0 + r) * kp + col] = diag ? X[r][col - j0] : 0.0;
    }
}

// Batched FP64 product C_p = alpha A_p B_p of s x s blocks (s a multiple of 32),
// pair p = blockIdx.z at A + p a_step etc.; one 32 x 32 tile of C_p per block.
struct PairGemm {
    const double* A;
    int64_t lda, a_step;
    const double* B;
    int64_t ldb, b_step;
    double* C;
    int64_t ldc, c_step;
    int s;
    double alpha;
};

__global__ void __launch_bounds__(256) blk_pair_gemm_kernel(const PairGemm g) {
    __shared__ double Ta[kTB][kTB + 1], Tb[kTB][kTB + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const double* A = g.A + (int64_t)blockIdx.z * g.a_step + (int64_t)blockIdx.y * kTB * g.lda;
    const double* B = g.B + (int64_t)blockIdx.z * g.b_step + (int64_t)blockIdx.x * kTB;
    double* C = g.C + (int64_t)blockIdx.z * g.c_step + (int64_t)blockIdx.y * kTB * g.ldc + (int64_t)blockIdx.x * kTB;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l0 = 0; l0 < g.s; l0 += kTB) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Ta[ty + 8 * q][tx] = A[(int64_t)(ty + 8 * q) * g.lda + l0 + tx];
            Tb[ty + 8 * q][tx] = B[(int64_t)(l0 + ty + 8 * q) * g.ldb + tx];
        }
        __syncthreads();
#pragma unroll 8
        for (int l = 0; l < kTB; ++l) {
            const double b = Tb[l][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(Ta[ty + 8 * q][l], b, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) C[(int64_t)(ty + 8 * q) * g.ldc + tx] = g.alpha * acc[q];
}

// Xinv (k x k FP32) = the leading block of Xp, zeros above the diagonal and in
// the rows of deflated columns.
__global__ void blk_out_kernel(const double* __restrict__ Xp, int kp, int k, const int* __restrict__ defl,
                               float* __restrict__ X) {
    const int64_t total = (int64_t)k * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / k), j = (int)(e % k);
        X[e] = (j <= i && !defl[i]) ? (float)Xp[(int64_t)i * kp + j] : 0.f;
    }
}

// the padded order: a power of two (the doubling levels then pair every block)
int kpad(int k) {
    int kp = kTB;
    while (kp < k) kp *= 2;
    return kp;
}

// L L^T = G (k x k FP64, ldg) and Xinv = L^{-1} (FP32); Lp, Xp hold kp^2 doubles,
// T kp^2 / 4, fl one double, defl kp ints; rel is the relative deflation threshold.
// Adds the number of kernels launched to *launches.
cudaError_t chol_inverse(const double* G, int ldg, int k, double rel, double* Lp, double* Xp, double* T, double* fl,
                         int* defl, float* Xinv, int* floored, cudaStream_t st, int* launches) {
    const int kp = kpad(k), nb = kp / kTB;
    int nl = 0;
    const int eb = (int)std::min<int64_t>(((int64_t)kp * kp + 255) / 256, 1024);
    blk_init_kernel<<<eb, 256, 0, st>>>(G, ldg, k, kp, Lp);
    blk_floor_kernel<<<1, 1024, 0, st>>>(G, ldg, k, fl);
    nl += 2;
    for (int J = 0; J < nb; ++J) {
        blk_potrf_trsm_kernel<<<nb - J, 1024, 0, st>>>(Lp, kp, J, G, ldg, k, rel, fl, defl, floored);
        ++nl;
        const int rem = nb - J - 1;
        if (rem > 0) {
            blk_syrk_kernel<<<rem * (rem + 1) / 2, 256, 0, st>>>(Lp, kp, J);
            ++nl;
        }
    }
    blk_inv_diag_kernel<<<nb, 1024, 0, st>>>(Lp, kp, Xp);
    ++nl;
    for (int s = kTB; s < kp; s *= 2) {
        const int pairs = kp / (2 * s);      // diagonal blocks of size 2s at o = p 2s
        // T_p = B A^{-1}: B = L[o+s.., o..], A^{-1} = X[o.., o..]
        PairGemm g1{Lp + (int64_t)s * kp, kp, (int64_t)2 * s * (kp + 1), Xp, kp, (int64_t)2 * s * (kp + 1),
                    T, s, (int64_t)s * s, s, 1.0};
        blk_pair_gemm_kernel<<<dim3(s / kTB, s / kTB, pairs), 256, 0, st>>>(g1);
        // X[o+s.., o..] = -C^{-1} T_p, C^{-1} = X[o+s.., o+s..]
        PairGemm g2{Xp + (int64_t)s * (kp + 1), kp, (int64_t)2 * s * (kp + 1), T, s, (int64_t)s * s,
                    Xp + (int64_t)s * kp, kp, (int64_t)2 * s * (kp + 1), s, -1.0};
        blk_pair_gemm_kernel<<<dim3(s / kTB, s / kTB, pairs), 256, 0, st>>>(g2);
        nl += 2;
    }
    blk_out_kernel<<<eb, 256, 0, st>>>(Xp, kp, k, defl, Xinv);
    ++nl;
    if (launches) *launches += nl;
    return cudaGetLastError();
}

// G (k x k, FP64) = C^T C for the first k columns of the r2 rows of the core C
// (FP64, row pitch ld): one 32 x 32 tile of G per block, 32-row slabs of C staged
// in shared memory.
__global__ void __launch_bounds__(256) gram64_kernel(const double* __restrict__ C, int64_t ld, int r2, int k,
                                                     double* __restrict__ G) {
    __shared__ double Ta[32][33], Tb[32][33];
    const int c1b = blockIdx.y * 32, c2b = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i0 = 0; i0 < r2; i0 += 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty + 8 * q;
            Ta[ty + 8 * q][tx] = (i < r2 && c1b + tx < k) ? C[(int64_t)i * ld + c1b + tx] : 0.0;
            Tb[ty + 8 * q][tx] = (i < r2 && c2b + tx < k) ? C[(int64_t)i * ld + c2b + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int ii = 0; ii < 32; ++ii) {
            const double b = Tb[ii][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(Ta[ii][ty + 8 * q], b, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int c1 = c1b + ty + 8 * q, c2 = c2b + tx;
        if (c1 < k && c2 < k) G[(int64_t)c1 * k + c2] = acc[q];
    }
}

// ---- FP32 CUDA-core GEMM: C(r, c) = sum_kk A(r, kk) B(kk, c) over the split's kk range.
// A(r, kk) = A[r sar + kk sak], B(kk, c) = B[kk sbk + c sbc], C(r, c) = C[z zstride + r ldc + c]
// for split z = blockIdx.z.  KA (KB): A (B) is contiguous along kk, else along r (c); each
// thread loads 8 elements of each 128 x 16 operand tile along the contiguous index, so a
// warp reads whole 64- or 128-byte runs.  Tiles are double-buffered in shared memory; each
// thread accumulates an 8 x 8 block (rows ty*4.., 64+ty*4..; columns tx*4.., 64+tx*4..).
constexpr int kGBM = 128, kGBN = 128, kGBK = 16, kGThreads = 256, kGPad = 4;

struct GemmArgs {
    const float* A;
    int64_t sar, sak;
    const float* B;
    int64_t sbk, sbc;
    float* C;
    int64_t ldc;
    int64_t M, N, K;
    int64_t kper;      // contraction length per split (a multiple of kGBK)
    int64_t zstride;   // floats between the partial outputs of consecutive splits
};

template <bool KA, bool KB>
__global__ void __launch_bounds__(kGThreads, 2) sgemm_kernel(const GemmArgs g) {
    __shared__ __align__(16) float As[2][kGBK][kGBM + kGPad];
    __shared__ __align__(16) float Bs[2][kGBK][kGBN + kGPad];
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int64_t r0 = (int64_t)blockIdx.y * kGBM, c0 = (int64_t)blockIdx.x * kGBN;
    const int64_t kb = (int64_t)blockIdx.z * g.kper;
    const int64_t ke = g.K < kb + g.kper ? g.K : kb + g.kper;
    // this thread's load coordinates within a tile
    const int arl = KA ? (t >> 4) : (t & 127), akl = KA ? (t & 15) : (t >> 7);
    const int bcl = KB ? (t >> 4) : (t & 127), bkl = KB ? (t & 15) : (t >> 7);
    float ra[8], rb[8];
    auto load = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int rl = KA ? arl + 16 * i : arl, kl = KA ? akl : akl + 2 * i;
            const int64_t r = r0 + rl, kk = k0 + kl;
            ra[i] = (r < g.M && kk < ke) ? g.A[r * g.sar + kk * g.sak] : 0.f;
            const int cl = KB ? bcl + 16 * i : bcl, kl2 = KB ? bkl : bkl + 2 * i;
            const int64_t c = c0 + cl, k2 = k0 + kl2;
            rb[i] = (c < g.N && k2 < ke) ? g.B[k2 * g.sbk + c * g.sbc] : 0.f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            As[buf][KA ? akl : akl + 2 * i][KA ? arl + 16 * i : arl] = ra[i];
            Bs[buf][KB ? bkl : bkl + 2 * i][KB ? bcl + 16 * i : bcl] = rb[i];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int64_t ntiles = ke > kb ? (ke - kb + kGBK - 1) / kGBK : 0;
    if (ntiles > 0) {
        load(kb);
        store(0);
        __syncthreads();
    }
    for (int64_t tt = 0; tt < ntiles; ++tt) {
        const int cur = (int)(tt & 1);
        if (tt + 1 < ntiles) load(kb + (tt + 1) * kGBK);
#pragma unroll
        for (int kk = 0; kk < kGBK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (tt + 1 < ntiles) store(cur ^ 1);
        __syncthreads();
    }
    float* C = g.C + (int64_t)blockIdx.z * g.zstride;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (r >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t c = c0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
            if (c < g.N) C[r * g.ldc + c] = acc[i][j];
        }
    }
}

// out(r, c) = sum over the splits z = 0, 1, ... of P[z zstride + r N + c], summed in
// FP64 in that order.
template <typename TO>
__global__ void reduce_parts_kernel(const float* __restrict__ P, int splits, int64_t zstride, int64_t M, int64_t N,
                                    TO* __restrict__ out, int64_t ldo) {
    const int64_t total = M * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / N, c = e % N;
        double acc = 0.0;
        for (int z = 0; z < splits; ++z) acc += (double)P[(int64_t)z * zstride + e];
        out[r * ldo + c] = (TO)acc;
    }
}

int g_qb_sms = 0;

int sm_count() {
    if (!g_qb_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_qb_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_qb_sms <= 0) g_qb_sms = 1;
    }
    return g_qb_sms;
}

// Splits of the contraction for an M x N output: enough blocks for two per SM,
// at least 512 contraction entries per split, at most `cap`.
int choose_splits(int64_t M, int64_t N, int64_t K, int cap) {
    const int64_t tiles = ((M + kGBM - 1) / kGBM) * ((N + kGBN - 1) / kGBN);
    const int64_t want = (2 * (int64_t)sm_count() + tiles - 1) / tiles;
    const int64_t by_len = std::max<int64_t>(1, K / 512);
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, by_len, (int64_t)cap}));
}

template <bool KA, bool KB>
cudaError_t gemm(const float* A, int64_t sar, int64_t sak, const float* B, int64_t sbk, int64_t sbc, float* C,
                 int64_t ldc, int64_t M, int64_t N, int64_t K, int splits, int64_t zstride, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    GemmArgs g{A, sar, sak, B, sbk, sbc, C, ldc, M, N, K, 0, zstride};
    const int64_t per = (K + splits - 1) / splits;
    g.kper = std::max<int64_t>(kGBK, (per + kGBK - 1) / kGBK * kGBK);
    const dim3 grid((unsigned)((N + kGBN - 1) / kGBN), (unsigned)((M + kGBM - 1) / kGBM), (unsigned)splits);
    sgemm_kernel<KA, KB><<<grid, kGThreads, 0, st>>>(g);
    return cudaGetLastError();
}

template <typename TO>
cudaError_t reduce_parts(const float* P, int splits, int64_t M, int64_t N, TO* out, int64_t ldo, cudaStream_t st) {
    const int64_t total = M * N;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * (int64_t)sm_count());
    reduce_parts_kernel<TO><<<blocks, 256, 0, st>>>(P, splits, M * N, M, N, out, ldo);
    return cudaGetLastError();
}

// Workspace carve-up (see qb_workspace_bytes)
struct QbWs {
    double *G64, *Lp, *Xp, *T, *fl;
    int* defl;
    float *Xinv, *W, *Q1, *part;    // W and Q1: rows x vpitch(k), 16-byte aligned rows
    uint16_t* qt;                   // the Q^T terms of the tensor-core product
    uint16_t* xt;                   // tensor cores: the three BF16 planes of L^-1 rows, per 128-row chunk
};

// Row pitch of W and Q1 (k rounded up to 8): 16-byte aligned rows for the tensor
// maps, and whole 8-column groups for the right-sketch kernel's output widths.
int64_t vpitch(int k) { return (k + 7) / 8 * 8; }
// The L^-1 plane chunks of the tensor-core products V (L^-1)^T: 128 output
// columns each, rows of xt_ld(k) contraction entries.
int64_t xt_ld(int k) { return (k + 63) / 64 * 64; }
size_t xt_chunk_elems(int k) { return (size_t)3 * 128 * (size_t)xt_ld(k); }
int xt_chunks(int k) { return (k + 127) / 128; }

constexpr int kPartCap = 128;       // largest split count of any CUDA-core product
constexpr size_t kTcPartFloats = (size_t)16 << 20;   // tensor-core product partials: 64 MB

int tc_part_cap(int64_t cols) { return (int)std::max<int64_t>(1, (int64_t)kTcPartFloats / (128 * cols)); }
// Relative deflation thresholds (pivot over the column's own squared norm): the
// core is FP64 but holds what FP32 A X resolves, about 1e-7 of a column's norm
// at the noise floor, so 1e-24 deflates only columns dependent far below that;
// W is FP32 and its Gram matrix sums FP32 products, so a column adding less than
// 1e-6 of its norm (pivot 1e-12) is dependent at FP32 resolution.
constexpr double kDeflPre = 1e-24;
constexpr double kDeflPass = 1e-12;

size_t part_floats_needed(int64_t rows, int64_t cols, int k, bool tensor) {
    // the Gram splits (k x k each) and the product's splits (k x cols each, or
    // 128 x cols each on the tensor cores)
    const int64_t sg = choose_splits(k, k, rows, kPartCap);
    const int64_t sb = choose_splits(k, cols, rows, kPartCap);
    const int64_t a = sg * (int64_t)k * k;
    const int64_t b = sb > 1 ? sb * (int64_t)k * cols : 0;
    const int64_t c = tensor ? (int64_t)tc_part_cap(cols) * 128 * cols : 0;
    return (size_t)std::max({a, b, c});
}

size_t ws_doubles(int k) {
    const size_t kp = (size_t)kpad(k);
    return (size_t)k * k + 2 * kp * kp + kp * kp / 4 + 2 + kp / 2;   // G64, Lp, Xp, T, fl (+ pad), defl
}

QbWs carve(void* ws, int64_t rows, int64_t cols, int k, bool tensor) {
    const size_t kp = (size_t)kpad(k);
    QbWs w;
    w.G64 = static_cast<double*>(ws);
    w.Lp = w.G64 + (size_t)k * k;
    w.Xp = w.Lp + kp * kp;
    w.T = w.Xp + kp * kp;
    w.fl = w.T + kp * kp / 4;
    w.defl = reinterpret_cast<int*>(w.fl + 2);
    w.Xinv = reinterpret_cast<float*>(w.G64 + ws_doubles(k));
    const uintptr_t wa = reinterpret_cast<uintptr_t>(w.Xinv + (size_t)k * k);
    w.W = reinterpret_cast<float*>((wa + 15) & ~(uintptr_t)15);
    w.Q1 = w.W + (size_t)rows * vpitch(k);
    w.part = w.Q1 + (size_t)rows * vpitch(k);
    // 16-byte aligned: the tensor maps of the product start here
    const uintptr_t q = reinterpret_cast<uintptr_t>(w.part + part_floats_needed(rows, cols, k, tensor));
    w.qt = reinterpret_cast<uint16_t*>((q + 15) & ~(uintptr_t)15);
    w.xt = w.qt + (tensor ? (size_t)3 * qb_tc_qt_rows(k) * (size_t)qb_tc_qt_ld(rows) : 0);
    return w;
}

}  // namespace

cudaError_t launch_select_rank(const double* sigma_scaled, int r1, int64_t n, double eps, double norm_a, int p,
                               int s, QbSelect* out, cudaStream_t st) {
    select_rank_kernel<<<1, 32, 0, st>>>(sigma_scaled, r1, n, eps, norm_a, p, s, out);
    return cudaGetLastError();
}

size_t qb_workspace_bytes(int64_t rows, int64_t cols, int k, bool tensor) {
    // the FP64 factorization buffers, the FP32 inverse (k x k), W and Q1 (rows x k
    // FP32), the split partials, the Q^T terms (tensor cores)
    const size_t qt = tensor ? sizeof(uint16_t) * 3 * (size_t)qb_tc_qt_rows(k) * (size_t)qb_tc_qt_ld(rows) : 0;
    const size_t xt = tensor ? sizeof(uint16_t) * xt_chunk_elems(k) * (size_t)xt_chunks(k) : 0;
    return sizeof(double) * ws_doubles(k) + sizeof(float) * ((size_t)k * k + (size_t)2 * rows * vpitch(k)) +
           sizeof(float) * part_floats_needed(rows, cols, k, tensor) + qt + xt + 256 + 32;
}

cudaError_t reduce_parts_f32(const float* part, int splits, int64_t M, int64_t N, float* out, int64_t ldo,
                             cudaStream_t st) {
    return reduce_parts<float>(part, splits, M, N, out, ldo, st);
}

cudaError_t reduce_parts_f64(const float* part, int splits, int64_t M, int64_t N, double* out, int64_t ldo,
                             cudaStream_t st) {
    return reduce_parts<double>(part, splits, M, N, out, ldo, st);
}

namespace {
// out (rows x k, pitch ldo, a multiple of 8 at least vpitch(k), 16-byte aligned) =
// V (rows x k, pitch ldv) (L^-1)^T on the tensor cores: the rows of L^-1 (Xinv, k x k)
// as three BF16 planes per 128 output columns, six products per K step; the
// columns [k, vpitch(k)) of out receive zeros.  Returns cudaErrorNotSupported when
// V does not suit the kernel (the caller then uses the CUDA-core tiles).
cudaError_t vlinv_tc(const float* V, int64_t ldv, int64_t rows, int k, const float* Xinv, uint16_t* xt, float* out,
                     int64_t ldo, int* err_flag, cudaStream_t st, int* launches) {
    MatView Vv;
    Vv.ptr = V;
    Vv.dtype = RE_F32;
    Vv.trans = false;
    Vv.rows = rows;
    Vv.cols = k;
    Vv.ld = ldv;
    if (!err_flag || !tc_supported(Vv) || (ldo % 8) != 0 || ldo < vpitch(k) ||
        (reinterpret_cast<uintptr_t>(out) & 15) != 0)
        return cudaErrorNotSupported;
    const int64_t ldt = xt_ld(k);
    cudaError_t e = cudaSuccess;
    for (int c0 = 0, ch = 0; c0 < k && e == cudaSuccess; c0 += 128, ++ch) {
        const int w = std::min(128, k - c0);
        const int s8 = (w + 7) / 8 * 8;                 // c0 + s8 <= vpitch(k) <= ldo
        const int nrows = tc_mma_n(s8);
        uint16_t* planes = xt + (size_t)ch * xt_chunk_elems(k);
        e = launch_rows_split3(Xinv, k, c0, w, k, nrows, ldt, planes, st);
        int nl = 0;
        if (e == cudaSuccess)
            e = launch_right_tc(Vv, planes, ldt, s8, out + c0, ldo, err_flag, st, &nl, 0, 3);
        if (launches) *launches += 1 + nl;
    }
    return e;
}
}  // namespace

cudaError_t launch_qb_precondition(const float* AX, int64_t sar, int64_t sak, int64_t rows, int64_t cols,
                                   const double* core, int64_t ld_core, int r2, int k, void* ws, int* floored,
                                   cudaStream_t st, int* launches, bool tensor, int* err_flag) {
    if (k <= 0 || k > 1024) return cudaErrorInvalidValue;
    QbWs w = carve(ws, rows, cols, k, tensor);
    // R_s^T R_s = C_k^T C_k (C_k = the first k columns of the r2 x s core), L = R_s^T
    const dim3 g64((unsigned)((k + 31) / 32), (unsigned)((k + 31) / 32));
    gram64_kernel<<<g64, 256, 0, st>>>(core, ld_core, r2, k, w.G64);
    if (launches) *launches += 1;
    cudaError_t e = chol_inverse(w.G64, k, k, kDeflPre, w.Lp, w.Xp, w.T, w.fl, w.defl, w.Xinv, floored, st, launches);
    if (e != cudaSuccess) return e;
    // W = (A X_k) R_s^{-1} = (A X_k) (L^{-1})^T: W(r, c) = sum_l AX(r, l) Xinv[c][l],
    // AX(r, l) at AX[r sar + l sak] (row-major, or the transposed planes of the
    // exact-product mode)
    const int64_t kp = vpitch(k);
    if (tensor && sak == 1) {
        e = vlinv_tc(AX, sar, rows, k, w.Xinv, w.xt, w.W, kp, err_flag, st, launches);
        if (e != cudaErrorNotSupported) return e;
    }
    e = sak == 1 ? gemm<true, true>(AX, sar, 1, w.Xinv, 1, k, w.W, kp, rows, k, k, 1, 0, st)
                 : gemm<false, true>(AX, sar, sak, w.Xinv, 1, k, w.W, kp, rows, k, k, 1, 0, st);
    if (launches) *launches += 1;
    return e;
}

cudaError_t launch_qb_orthonormalise(int64_t rows, int64_t cols, int k, float* Q, int64_t ldq, void* ws,
                                     int* floored, cudaStream_t st, int* launches, bool tensor, int* err_flag) {
    QbWs w = carve(ws, rows, cols, k, tensor);
    const int64_t kp = vpitch(k);
    // two Cholesky-QR passes: G = V^T V, V <- V (L^{-1})^T
    float* V = w.W;
    const int splits = choose_splits(k, k, rows, kPartCap);
    cudaError_t e = cudaSuccess;
    MatView Vv;
    Vv.dtype = RE_F32;
    Vv.trans = false;
    Vv.rows = rows;
    Vv.cols = k;
    Vv.ld = kp;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        Vv.ptr = V;
        // partial Gram matrices over row ranges, summed in FP64: on the tensor cores
        // as the product V^T V (both factors in three BF16 terms, six products)
        if (tensor && err_flag && qb_tc_supported(Vv)) {
            e = launch_qt_split(V, kp, rows, k, w.qt, st);
            int nl = 1;
            const int64_t tiles = (k + 127) / 128, kchunks = (rows + 63) / 64;
            const int ts = qb_tc_splits(tiles, kchunks, tc_part_cap(k));
            for (int c0 = 0; c0 < k && e == cudaSuccess; c0 += 128) {
                const int kq = std::min(128, k - c0);
                e = launch_qb_product_tc(Vv, w.qt, k, c0, kq, nullptr, 0, w.part, ts, err_flag, st,
                                         w.G64 + (size_t)c0 * k, k);
                nl += 2;
            }
            if (launches) *launches += nl;
        } else {
            e = gemm<false, false>(V, 1, kp, V, kp, 1, w.part, k, k, k, rows, splits, (int64_t)k * k, st);
            if (e == cudaSuccess) e = reduce_parts<double>(w.part, splits, k, k, w.G64, k, st);
            if (launches) *launches += 2;
        }
        if (e == cudaSuccess)
            e = chol_inverse(w.G64, k, k, kDeflPass, w.Lp, w.Xp, w.T, w.fl, w.defl, w.Xinv, floored, st, launches);
        if (e != cudaSuccess) break;
        // V (L^-1)^T: pass 0 into Q1; pass 1 into Q, through W (free after pass 0) on
        // the tensor cores, whose output rows are padded to whole 8-column groups
        float* tout = pass == 0 ? w.Q1 : w.W;
        cudaError_t et = tensor ? vlinv_tc(V, kp, rows, k, w.Xinv, w.xt, tout, kp, err_flag, st, launches)
                                : cudaErrorNotSupported;
        if (et == cudaSuccess && pass == 1) {
            et = cudaMemcpy2DAsync(Q, sizeof(float) * ldq, w.W, sizeof(float) * kp, sizeof(float) * k, rows,
                                   cudaMemcpyDeviceToDevice, st);
        } else if (et == cudaErrorNotSupported) {
            float* out = pass == 0 ? w.Q1 : Q;
            const int64_t ldo = pass == 0 ? kp : ldq;
            et = gemm<true, true>(V, kp, 1, w.Xinv, 1, k, out, ldo, rows, k, k, 1, 0, st);
            if (launches) *launches += 1;
        }
        e = et;
        V = w.Q1;
    }
    return e;
}

cudaError_t launch_qb_product(const MatView& A, const float* Q, int64_t ldq, int k, float* B, int64_t ldb, void* ws,
                              bool tensor, int* err_flag, cudaStream_t st, int* launches) {
    if (A.dtype != RE_F32) return cudaErrorInvalidValue;
    const float* Ap = static_cast<const float*>(A.ptr);
    const int64_t M = A.rows, N = A.cols;
    if (tensor && qb_tc_supported(A)) {
        // B = Q^T A on the tensor cores: the three BF16 terms of Q^T once, then one
        // launch per 128 columns of Q (each reads A once)
        QbWs w = carve(ws, M, N, k, true);
        cudaError_t e = launch_qt_split(Q, ldq, M, k, w.qt, st);
        int nl = 1;
        const int64_t tiles = (N + 127) / 128, kchunks = (M + 63) / 64;
        const int splits = qb_tc_splits(tiles, kchunks, tc_part_cap(N));
        for (int c0 = 0; c0 < k && e == cudaSuccess; c0 += 128) {
            const int kq = std::min(128, k - c0);
            e = launch_qb_product_tc(A, w.qt, k, c0, kq, B + (size_t)c0 * ldb, ldb, w.part, splits, err_flag, st);
            nl += splits > 1 ? 2 : 1;
        }
        if (launches) *launches += nl;
        return e;
    }
    QbWs w = carve(ws, M, N, k, false);
    const int splits = choose_splits(k, N, M, kPartCap);
    float* out = splits > 1 ? w.part : B;
    const int64_t ldo = splits > 1 ? N : ldb;
    const int64_t zs = (int64_t)k * N;
    // B(c, j) = sum_i Q[i][c] A_o(i, j); A_o(i, j) = A[i][j], or A[j][i] when the view is transposed
    cudaError_t e = A.trans ? gemm<false, true>(Q, 1, ldq, Ap, 1, A.ld, out, ldo, k, N, M, splits, zs, st)
                            : gemm<false, false>(Q, 1, ldq, Ap, A.ld, 1, out, ldo, k, N, M, splits, zs, st);
    if (launches) *launches += 1;
    if (e == cudaSuccess && splits > 1) {
        e = reduce_parts<float>(w.part, splits, k, N, B, ldb, st);
        if (launches) *launches += 1;
    }
    return e;
}

}  // namespace re
