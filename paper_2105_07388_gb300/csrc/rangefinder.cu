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
// factorizations (Cholesky, triangular inverse; k <= 512) run in one CTA in
// FP64; every product is a plain cuBLAS GEMM (FP64 for the core's Gram, FP32
// otherwise, pedantic math mode: no reduced-precision tensor paths).
#include <cmath>

#include <cublas_v2.h>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kSmallThreads = 1024;

__global__ void select_rank_kernel(const double* __restrict__ sig, int r1, int64_t n, double eps, double norm_a,
                                   int p, int s, QbSelect* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double ref = norm_a > 0.0 ? norm_a : (r1 > 0 ? sig[0] : 0.0);
    // A has only n singular values: a sketch wider than n trusts at most n of them
    const int re = (int)(n < (int64_t)r1 ? n : (int64_t)r1);
    const double last = re > 0 ? sig[re - 1] : 0.0;
    // T(r) = sum_{j>r} sigma^_j^2, accumulated from the tail: T(re) = (n - re) sigma^_{re}^2
    double T = (double)(n - re) * last * last;
    int best = -1;
    double best_bound = 0.0;
    for (int r = re; r >= 0; --r) {
        if (r < re) T += sig[r] * sig[r];
        const double bound = sqrt(1.0 + (double)r / (p - 1.0)) * sqrt(T);
        if (bound <= eps * ref) {
            best = r;                     // walking down: the last hit is the smallest r
            best_bound = bound;
        }
    }
    out->r = best;
    // k = min(r + p, n) columns factor A exactly once the sketch covers all n
    // singular values, so the criterion is met when those k columns are sketched
    const int64_t k = (int64_t)best + p < n ? (int64_t)best + p : n;
    out->met = (best >= 0 && k <= s) ? 1 : 0;
    out->bound = best_bound;
    out->norm_a = ref;
}

// The lower triangle of the k x k row-major G (FP64, or FP32 widened) is copied
// to L and factored in place, G = L L^T.  A pivot not above 1e-30 of the largest
// diagonal entry (an exactly singular Gram matrix) is raised to it, 1 when the
// whole matrix is zero, and *floored is set.
template <typename TG>
__global__ void __launch_bounds__(kSmallThreads) chol_lower_kernel(const TG* __restrict__ G, int ldg, double* L,
                                                                  int k, int* floored) {
    __shared__ double s_inv, s_floor;
    const int tid = threadIdx.x;
    for (int64_t e = tid; e < (int64_t)k * k; e += blockDim.x) {
        const int i = (int)(e / k), l = (int)(e % k);
        L[e] = l <= i ? (double)G[(int64_t)i * ldg + l] : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, L[(int64_t)i * k + i]);
        s_floor = mx > 0.0 ? mx * 1e-30 : 1.0;      // an all-zero Gram matrix (A X_k = 0) factors as L = I
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            double d = L[(int64_t)j * k + j];
            if (!(d > s_floor)) {
                d = s_floor;
                if (floored) *floored = 1;
            }
            const double sd = sqrt(d);
            L[(int64_t)j * k + j] = sd;
            s_inv = 1.0 / sd;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < k; i += blockDim.x) L[(int64_t)i * k + j] *= s_inv;
        __syncthreads();
        for (int i = j + 1 + tid; i < k; i += blockDim.x) {
            const double lij = L[(int64_t)i * k + j];
            for (int l = j + 1; l <= i; ++l) L[(int64_t)i * k + l] -= lij * L[(int64_t)l * k + j];
        }
        __syncthreads();
    }
}

// X = L^{-1} (lower triangular, FP64 forward substitution, one thread per column),
// written as FP32 with zeros above the diagonal.
__global__ void __launch_bounds__(kSmallThreads) tri_inv_lower_kernel(const double* __restrict__ L, int k,
                                                                     double* __restrict__ work,
                                                                     float* __restrict__ X) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        double* x = work + (int64_t)j * k;           // column j of L^{-1}, rows j .. k-1
        x[j] = 1.0 / L[(int64_t)j * k + j];
        for (int i = j + 1; i < k; ++i) {
            double acc = 0.0;
            for (int l = j; l < i; ++l) acc = fma(L[(int64_t)i * k + l], x[l], acc);
            x[i] = -acc / L[(int64_t)i * k + i];
        }
        for (int i = 0; i < k; ++i) X[(int64_t)i * k + j] = i < j ? 0.f : (float)x[i];
    }
}

// Row-major C (mr x nc) = op_a(A) op_b(B) through column-major cuBLAS (the row-major
// matrices are the transposes cuBLAS sees; C^T = op_b(B)^T op_a(A)^T).
cublasStatus_t sgemm_rm(cublasHandle_t hb, bool ta, bool tb, int mr, int nc, int kk, const float* A, int64_t lda,
                        const float* B, int64_t ldb, float* C, int64_t ldc) {
    const float one = 1.f, zero = 0.f;
    return cublasSgemm(hb, tb ? CUBLAS_OP_T : CUBLAS_OP_N, ta ? CUBLAS_OP_T : CUBLAS_OP_N, nc, mr, kk, &one, B,
                       (int)ldb, A, (int)lda, &zero, C, (int)ldc);
}

cudaError_t cublas_err(cublasStatus_t s) { return s == CUBLAS_STATUS_SUCCESS ? cudaSuccess : cudaErrorUnknown; }

}  // namespace

cudaError_t launch_select_rank(const double* sigma_scaled, int r1, int64_t n, double eps, double norm_a, int p,
                               int s, QbSelect* out, cudaStream_t st) {
    select_rank_kernel<<<1, 32, 0, st>>>(sigma_scaled, r1, n, eps, norm_a, p, s, out);
    return cudaGetLastError();
}

size_t qb_workspace_bytes(int64_t rows, int k) {
    // W and Q1 (rows x k FP32), two FP32 k x k (Gram, inverse), two FP64 k x k (L, work)
    return sizeof(float) * ((size_t)2 * rows * k + (size_t)2 * k * k) + sizeof(double) * (size_t)2 * k * k + 256;
}

cudaError_t launch_qb_factor(void* cublas, const MatView& A, const float* AX, int64_t ldax, const double* core,
                             int64_t ld_core, int r2, int k, float* Q, int64_t ldq, float* B, int64_t ldb, void* ws,
                             int* floored, cudaStream_t st) {
    if (A.dtype != RE_F32 || k <= 0 || k > 1024) return cudaErrorInvalidValue;
    cublasHandle_t hb = static_cast<cublasHandle_t>(cublas);
    if (cublasSetStream(hb, st) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    if (cublasSetMathMode(hb, CUBLAS_PEDANTIC_MATH) != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    const int64_t M = A.rows;
    float* W = static_cast<float*>(ws);
    float* Q1 = W + (size_t)M * k;
    float* G32 = Q1 + (size_t)M * k;
    float* Xinv = G32 + (size_t)k * k;
    double* L = reinterpret_cast<double*>(Xinv + (size_t)k * k);   // 2 M k + 2 k^2 floats: 8-byte aligned
    double* work = L + (size_t)k * k;
    double* G64 = work;                               // the core's Gram, consumed before work is needed
    // R_s: Cholesky of the core's Gram C_k^T C_k (C_k = the first k columns of the r2 x s core)
    {
        const double one = 1.0, zero = 0.0;
        cublasStatus_t cs = cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, k, k, r2, &one, core, (int)ld_core, core,
                                        (int)ld_core, &zero, G64, k);
        if (cs != CUBLAS_STATUS_SUCCESS) return cublas_err(cs);
    }
    chol_lower_kernel<double><<<1, kSmallThreads, 0, st>>>(G64, k, L, k, floored);
    tri_inv_lower_kernel<<<1, kSmallThreads, 0, st>>>(L, k, work, Xinv);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // W = (A X_k) R_s^{-1} = (A X_k) (L^{-1})^T
    cublasStatus_t cs = sgemm_rm(hb, false, true, (int)M, k, k, AX, ldax, Xinv, k, W, k);
    if (cs != CUBLAS_STATUS_SUCCESS) return cublas_err(cs);
    // two Cholesky-QR passes: G = V^T V, V <- V (L^{-1})^T
    const float* V = W;
    for (int pass = 0; pass < 2; ++pass) {
        float* out = pass == 0 ? Q1 : Q;
        const int64_t ldo = pass == 0 ? k : ldq;
        cs = sgemm_rm(hb, true, false, k, k, (int)M, V, k, V, k, G32, k);
        if (cs != CUBLAS_STATUS_SUCCESS) return cublas_err(cs);
        chol_lower_kernel<float><<<1, kSmallThreads, 0, st>>>(G32, k, L, k, floored);
        tri_inv_lower_kernel<<<1, kSmallThreads, 0, st>>>(L, k, work, Xinv);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cs = sgemm_rm(hb, false, true, (int)M, k, k, V, k, Xinv, k, out, ldo);
        if (cs != CUBLAS_STATUS_SUCCESS) return cublas_err(cs);
        V = Q1;
    }
    // B = Q^T A_oriented (k x cols): A_oriented is A (row-major) or A^T when transposed
    cs = sgemm_rm(hb, true, A.trans, k, (int)A.cols, (int)M, Q, ldq, static_cast<const float*>(A.ptr), A.ld, B,
                  ldb);
    return cublas_err(cs);
}

}  // namespace re
