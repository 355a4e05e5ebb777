// Singular values of the small sketched core Y*A*X (Algorithm 1 step 7) and the
// read-off of the eps-rank (step 8).
//
// Step 7 uses one-sided (Hestenes) Jacobi: pairs of columns are rotated until
// every pair is orthogonal to working precision; the singular values are then
// the column norms.  It never forms the Gram matrix (which would square the
// condition number and lose the small singular values the rank read-off
// depends on).  Pairs are scheduled by the round-robin (circle) ordering, so
// the s/2 rotations of a round are independent and run on separate warps of
// one CTA.  The working copy lives in shared memory when it fits and in a
// global workspace otherwise.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kSvdThreads = 512;
constexpr int kMaxSweeps = 40;

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr double u = 5.9604644775390625e-08; };
template <> struct Eps<double> { static constexpr double u = 1.1102230246251565e-16; };

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One-sided Jacobi on the column-major rows x cols matrix W (leading dim ldw),
// executed by the whole CTA.  Returns the number of sweeps used.
template <typename T>
__device__ int jacobi_sweeps(T* W, int rows, int cols, int ldw, int* s_flag) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int P = cols + (cols & 1);
    const T tol = (T)(4.0 * Eps<T>::u * sqrt((double)rows));
    int sweep = 0;
    for (; sweep < kMaxSweeps; ++sweep) {
        if (threadIdx.x == 0) *s_flag = 0;
        __syncthreads();
        for (int t = 0; t < P - 1; ++t) {
            for (int k = warp; k < P / 2; k += nwarps) {
                const int i1 = k, i2 = P - 1 - k;
                const int c1 = (i1 == 0) ? 0 : 1 + (i1 - 1 + t) % (P - 1);
                const int c2 = (i2 == 0) ? 0 : 1 + (i2 - 1 + t) % (P - 1);
                const int p = min(c1, c2), q = max(c1, c2);
                if (q >= cols) continue;
                T* a = W + (int64_t)p * ldw;
                T* b = W + (int64_t)q * ldw;
                T al = 0, be = 0, ga = 0;
                for (int i = lane; i < rows; i += 32) {
                    const T x = a[i], y = b[i];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga == (T)0 || !(fabs(ga) > tol * sqrt(al) * sqrt(be))) continue;
                const T zeta = (be - al) / (ga + ga);
                T tt;
                if (fabs(zeta) > (T)1e15) {
                    tt = (T)0.5 / zeta;
                } else {
                    tt = copysign((T)1, zeta) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
                }
                const T c = (T)1 / sqrt((T)1 + tt * tt);
                const T sn = c * tt;
                for (int i = lane; i < rows; i += 32) {
                    const T x = a[i], y = b[i];
                    a[i] = c * x - sn * y;
                    b[i] = sn * x + c * y;
                }
                if (lane == 0) *s_flag = 1;
            }
            __syncthreads();
        }
        const int any = *s_flag;
        __syncthreads();
        if (!any) break;
    }
    return sweep;
}

// Column norms (accumulated in FP64), sorted descending into sigma_out.
template <typename T>
__device__ void norms_sorted(const T* W, int rows, int cols, int ldw, double* s_norm,
                             double* sigma_out) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    for (int j = warp; j < cols; j += nwarps) {
        double acc = 0.0;
        const T* a = W + (int64_t)j * ldw;
        for (int i = lane; i < rows; i += 32) {
            const double x = (double)a[i];
            acc = fma(x, x, acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) s_norm[j] = sqrt(acc);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < cols; j += blockDim.x) {
        const double v = s_norm[j];
        int rank = 0;
        for (int i = 0; i < cols; ++i) {
            const double w = s_norm[i];
            rank += (w > v) || (w == v && i < j);
        }
        sigma_out[rank] = v;
    }
}

// Whole step 7 for one core: copy (checking finiteness), Jacobi, norms.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(kSvdThreads) core_sigma_kernel(const double* __restrict__ core,
                                                                 int r2, int s, int64_t ld,
                                                                 T* __restrict__ gW,
                                                                 double* __restrict__ sigma,
                                                                 int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    __shared__ int s_bad;
    __shared__ double s_norm[512];
    T* W = SMEM ? reinterpret_cast<T*>(smem) : gW;
    const int ldw = r2;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    int bad = 0;
    for (int64_t idx = threadIdx.x; idx < (int64_t)r2 * s; idx += blockDim.x) {
        const int i = (int)(idx / s), j = (int)(idx % s);
        const double v = core[(int64_t)i * ld + j];
        bad |= !isfinite(v);
        W[(int64_t)j * ldw + i] = (T)v;
    }
    if (bad) s_bad = 1;
    __syncthreads();
    if (s_bad) {
        for (int j = threadIdx.x; j < s; j += blockDim.x) sigma[j] = nan("");
        if (threadIdx.x == 0) *status = RE_ERR_NONFINITE;
        return;
    }
    jacobi_sweeps<T>(W, r2, s, ldw, &s_flag);
    norms_sorted<T>(W, r2, s, ldw, s_norm, sigma);
    if (threadIdx.x == 0) *status = RE_OK;
}

// Step 8 (device): scaled sigma, threshold rank, gap index.
__global__ void readoff_kernel(const double* __restrict__ sigma, int r1, double scale, double eps,
                               double norm_a, const int* __restrict__ status_in,
                               DevReadoff* __restrict__ out, double* __restrict__ sigma_scaled) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevReadoff r;
    r.status = status_in ? *status_in : RE_OK;
    r.pad = 0;
    for (int i = 0; i < r1; ++i) sigma_scaled[i] = sigma[i] * scale;
    const double ref = norm_a > 0.0 ? norm_a : sigma_scaled[0];
    r.tau = eps * ref;
    r.rank = -1;
    for (int i = 0; i < r1; ++i) {
        if (sigma_scaled[i] <= r.tau) {
            r.rank = i;
            break;
        }
    }
    int gi = r1 >= 1 ? 1 : 0;
    double gr = r1 >= 2 ? -1.0 : 1.0;
    for (int i = 1; i < r1; ++i) {
        const double a = sigma_scaled[i - 1], b = sigma_scaled[i];
        double ratio;
        if (b > 0.0) ratio = a / b;
        else if (a > 0.0) ratio = INFINITY;
        else ratio = 1.0;
        if (ratio > gr) {
            gr = ratio;
            gi = i;
        }
    }
    r.gap_index = gi;
    r.gap_ratio = gr;
    *out = r;
}

template <typename T>
size_t smem_bytes(int r2, int s) { return sizeof(T) * (size_t)r2 * s; }

constexpr size_t kSmemLimit = 200 * 1024;

}  // namespace

size_t svd_workspace_bytes(int r2, int s) { return sizeof(float) * (size_t)r2 * s + 256; }

cudaError_t launch_core_sigma(const double* core, int r2, int s, int64_t ld, void* ws,
                              double* sigma, int* status, cudaStream_t st) {
    if (s <= 0) return cudaSuccess;
    const size_t sm = smem_bytes<float>(r2, s);
    if (sm <= kSmemLimit) {
        auto k = core_sigma_kernel<float, true>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k<<<1, kSvdThreads, sm, st>>>(core, r2, s, ld, nullptr, sigma, status);
    } else {
        core_sigma_kernel<float, false><<<1, kSvdThreads, 0, st>>>(core, r2, s, ld,
                                                                    static_cast<float*>(ws), sigma,
                                                                    status);
    }
    return cudaGetLastError();
}

cudaError_t launch_readoff(const double* sigma, int r1, double scale, double eps, double norm_a,
                           const int* status_in, DevReadoff* out, double* sigma_scaled,
                           cudaStream_t st) {
    readoff_kernel<<<1, 32, 0, st>>>(sigma, r1, scale, eps, norm_a, status_in, out, sigma_scaled);
    return cudaGetLastError();
}

}  // namespace re
