// Singular values of the small sketched core Y*A*X (Algorithm 1 step 7) and the
// read-off of the eps-rank (step 8).
//
// Step 7: the r2 x s core is scaled by a power of two (exact), reduced by a
// Householder QR to its s x s triangular factor R (sigma(core) = sigma(R)), and
// one-sided (Hestenes) Jacobi is run on the columns of R^T until every pair is
// orthogonal to working precision; the singular values are the column norms.
// The QR step is the classical preconditioner for one-sided Jacobi (the rows of
// R are graded, so Jacobi on R^T converges in a few sweeps).  The Gram matrix is
// never formed (it would square the condition number and lose the small
// singular values the read-off depends on).  Pairs are scheduled by the
// round-robin (circle) ordering, so the rotations of a round are independent
// and run on separate warps.
//
// Arithmetic is FP32: on GB300 FP64 runs at about 1/57 of the FP32 rate, and the
// sketch itself is accumulated in FP32, so FP32 rotations (absolute error about
// 1e-5 sigma_1 at s = 512) keep the whole path consistent.  Rotations whose
// off-diagonal term is below (1e-7 sigma_1)^2 are skipped: they cannot move any
// singular value by more than 1e-7 sigma_1, far below the FP32 noise floor.
//
// Small cores (r2 s + s^2 floats fit in shared memory) use one CTA; larger cores
// use a cluster of 8 or 16 CTAs: the QR is column-cyclic with the Householder
// vector broadcast over distributed shared memory, and Jacobi is blocked (two
// column blocks per CTA, blocks rotating through the cluster each round).
#include <cfloat>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

namespace cg = cooperative_groups;

constexpr int kSvdThreads = 512;
constexpr int kMaxSweeps = 40;
constexpr float kU = 5.9604644775390625e-08f;        // 2^-24
constexpr float kAbsFloor = 1e-14f;                  // (1e-7)^2 of max column norm^2
// A sweep whose largest rotated |cos| is below kStopFactor * u * sqrt(n) only
// rotated pairs at the FP32 rounding level of the dot products: stop there.
constexpr float kStopFactor = 32.f;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Lanes per column pair in a Jacobi rotation: a warp works on four pairs at once
// (three-level reductions, four independent dependency chains).
constexpr int kG = 8;

__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = kG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Jacobi rotation of columns a, b (length n) by a group of kG lanes; returns 1 if
// this group rotated.  Every lane of the warp must call it (the reductions use
// full-warp shuffles); inactive groups pass active = false.
// n is a multiple of kG (columns are zero padded); the four groups of a warp
// start their traversal kG*g elements apart so that, with column strides that
// are multiples of 32 floats, they touch disjoint shared-memory banks.
__device__ __forceinline__ int rotate_pair(bool active, float* a, float* b, int n, float tol,
                                           float floor_abs, float* meas) {
    const int gl = threadIdx.x & (kG - 1);
    const int J = n / kG;
    const int j0 = J > 0 ? ((threadIdx.x >> 3) & 3) % J : 0;
    float al = 0.f, be = 0.f, ga = 0.f;
    if (active) {
        for (int jj = 0, j = j0; jj < J; ++jj, j = (j + 1 == J) ? 0 : j + 1) {
            const int i = j * kG + gl;
            const float x = a[i], y = b[i];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
        }
    }
    al = group_sum(al);
    be = group_sum(be);
    ga = group_sum(ga);
    const float ag = fabsf(ga);
    if (!active || !(ag > tol * sqrtf(al) * sqrtf(be)) || !(ag > floor_abs)) return 0;
    *meas = ag / (sqrtf(al) * sqrtf(be));
    const float zeta = (be - al) / (ga + ga);
    const float tt = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                         : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
    const float c = 1.f / sqrtf(1.f + tt * tt);
    const float sn = c * tt;
    for (int jj = 0, j = j0; jj < J; ++jj, j = (j + 1 == J) ? 0 : j + 1) {
        const int i = j * kG + gl;
        const float x = a[i], y = b[i];
        a[i] = fmaf(c, x, -sn * y);
        b[i] = fmaf(sn, x, c * y);
    }
    return 1;
}

// FP64-accumulated norm of a length-n column (one warp).
__device__ __forceinline__ double col_norm(const float* a, int n) {
    const int lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int i = lane; i < n; i += 32) {
        const double x = (double)a[i];
        acc = fma(x, x, acc);
    }
    return sqrt(warp_sum(acc));
}

// Descending rank sort of s_norm[0..n) into out (scaled by `scale`).
__device__ void sort_desc(const double* s_norm, int n, double scale, double* out) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = s_norm[j];
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            const double w = s_norm[i];
            rank += (w > v) || (w == v && i < j);
        }
        out[rank] = v * scale;
    }
}

// Householder reflector of x[0..L) (one warp): x[1..) becomes v (v[0] = 1
// implicit), x[0] becomes beta; returns tau with H = I - tau v v^T.
__device__ __forceinline__ float householder(float* x, int L) {
    const int lane = threadIdx.x & 31;
    float ss = 0.f;
    for (int i = 1 + lane; i < L; i += 32) ss = fmaf(x[i], x[i], ss);
    ss = warp_sum(ss);
    const float x0 = x[0];
    float tau = 0.f, beta = x0;
    if (ss > 0.f) {
        const float nrm = sqrtf(fmaf(x0, x0, ss));
        beta = -copysignf(nrm, x0);
        tau = (beta - x0) / beta;
        const float scale = 1.f / (x0 - beta);
        __syncwarp();
        for (int i = 1 + lane; i < L; i += 32) x[i] *= scale;
    }
    __syncwarp();
    if (lane == 0) x[0] = beta;
    __syncwarp();
    return tau;
}

// ---------------------------------------------------------------------------
// One CTA per core: core -> shared memory (column-major, scaled), QR in place,
// R^T -> second region, Jacobi on R^T, norms.  blockIdx.x selects the core
// (core_stride / sigma_stride apart) so one launch serves a batch.
__global__ void __launch_bounds__(kSvdThreads) core_sigma_cta_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, int64_t core_stride,
    double* __restrict__ sigma, int64_t sigma_stride, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    core += (int64_t)blockIdx.x * core_stride;
    sigma += (int64_t)blockIdx.x * sigma_stride;
    const int sp = (s + 31) / 32 * 32;                  // padded column length of R^T
    float* W = reinterpret_cast<float*>(smem);          // r2 x s, column-major
    float* Rt = W + (size_t)r2 * s;                     // sp x s, column c = row c of R
    __shared__ double s_norm[512];
    __shared__ float s_tau, s_red[32];
    __shared__ int s_bad, s_flag;
    __shared__ unsigned int s_meas;
    __shared__ unsigned long long s_dmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    // power-of-two scale: largest |entry| -> [0.5, 1)
    if (tid == 0) {
        s_bad = 0;
        s_dmax = 0ull;
    }
    __syncthreads();
    double mx = 0.0;
    int bad = 0;
    for (int64_t idx = tid; idx < (int64_t)r2 * s; idx += blockDim.x) {
        const double v = core[(idx / s) * ld + idx % s];
        bad |= !isfinite(v);
        mx = fmax(mx, fabs(v));
    }
    if (bad) s_bad = 1;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && isfinite(mx)) atomicMax(&s_dmax, (unsigned long long)__double_as_longlong(mx));
    __syncthreads();
    if (s_bad) {
        for (int j = tid; j < s; j += blockDim.x) sigma[j] = nan("");
        if (tid == 0) status[blockIdx.x] = RE_ERR_NONFINITE;
        return;
    }
    int e2 = 0;
    const double dmax = __longlong_as_double((long long)s_dmax);
    if (dmax > 0.0) frexp(dmax, &e2);
    const double down = ldexp(1.0, -e2), up = ldexp(1.0, e2);
    for (int64_t idx = tid; idx < (int64_t)r2 * s; idx += blockDim.x) {
        const int i = (int)(idx / s), j = (int)(idx % s);
        W[(size_t)j * r2 + i] = (float)(core[(int64_t)i * ld + j] * down);
    }
    __syncthreads();

    // Householder QR: column k's reflector, then the trailing columns
    for (int k = 0; k < s; ++k) {
        float* colk = W + (size_t)k * r2 + k;
        if (warp == 0) {
            const float tau = householder(colk, r2 - k);
            if (lane == 0) s_tau = tau;
        }
        __syncthreads();
        const float tau = s_tau;
        if (tau != 0.f) {
            for (int j = k + 1 + warp; j < s; j += nwarps) {
                float* cj = W + (size_t)j * r2 + k;
                float w = 0.f;
                for (int i = lane; i < r2 - k; i += 32) w = fmaf(i == 0 ? 1.f : colk[i], cj[i], w);
                w = warp_sum(w) * tau;
                for (int i = lane; i < r2 - k; i += 32) cj[i] = fmaf(-w, i == 0 ? 1.f : colk[i], cj[i]);
            }
        }
        __syncthreads();
    }
    // R^T: column c of Rt = row c of R = W[j][c] for j >= c
    for (int64_t idx = tid; idx < (int64_t)s * sp; idx += blockDim.x) {
        const int c = (int)(idx / sp), j = (int)(idx % sp);
        Rt[(size_t)c * sp + j] = (j >= c && j < s) ? W[(size_t)j * r2 + c] : 0.f;
    }
    __syncthreads();

    // Jacobi on R^T (s x s)
    const int P = s + (s & 1);
    const float tol = 4.f * kU * sqrtf((float)s);
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        float amax = 0.f;
        for (int j = warp; j < s; j += nwarps) {
            float a = 0.f;
            for (int i = lane; i < sp; i += 32) a = fmaf(Rt[(size_t)j * sp + i], Rt[(size_t)j * sp + i], a);
            amax = fmaxf(amax, warp_sum(a));
        }
        if (lane == 0) s_red[warp] = amax;
        if (tid == 0) {
            s_flag = 0;
            s_meas = 0u;
        }
        __syncthreads();
        if (warp == 0) {
            const float v = warp_max(lane < nwarps ? s_red[lane] : 0.f);
            if (lane == 0) s_red[0] = v;
        }
        __syncthreads();
        const float floor_abs = kAbsFloor * s_red[0];
        const int grp = tid / kG, ngrp = blockDim.x / kG;
        for (int t = 0; t < P - 1; ++t) {
            for (int base = 0; base < P / 2; base += ngrp) {
                const int q = base + grp;
                int p = 0, qq = 0;
                bool act = q < P / 2;
                if (act) {
                    const int i1 = q, i2 = P - 1 - q;
                    const int c1 = (i1 == 0) ? 0 : 1 + (i1 - 1 + t) % (P - 1);
                    const int c2 = (i2 == 0) ? 0 : 1 + (i2 - 1 + t) % (P - 1);
                    p = min(c1, c2);
                    qq = max(c1, c2);
                    act = qq < s;
                }
                float meas = 0.f;
                if (rotate_pair(act, Rt + (size_t)p * sp, Rt + (size_t)qq * sp, sp, tol, floor_abs, &meas) &&
                    (tid & (kG - 1)) == 0) {
                    s_flag = 1;
                    atomicMax(&s_meas, __float_as_uint(meas));
                }
            }
            __syncthreads();
        }
        const int any = s_flag;
        const float worst = __uint_as_float(s_meas);
        __syncthreads();
        if (!any || worst < kStopFactor * kU * sqrtf((float)s)) {
            if (tid == 0 && blockIdx.x == 0 && sigma_stride == 0) status[2] = sweep + 1;
            break;
        }
        if (tid == 0 && blockIdx.x == 0 && sigma_stride == 0) status[2] = sweep + 1;
    }
    for (int j = warp; j < s; j += nwarps) {
        const double nv = col_norm(Rt + (size_t)j * sp, sp);
        if (lane == 0) s_norm[j] = nv;
    }
    __syncthreads();
    sort_desc(s_norm, s, up, sigma);
    if (tid == 0) status[blockIdx.x] = RE_OK;
}

// ---------------------------------------------------------------------------
// Cluster version.  Column j of the core lives in CTA j % CL (local column j / CL).
constexpr int kPullRegs = 32;       // per-thread staging for a block exchange

template <int CL>
__global__ void __launch_bounds__(kSvdThreads, 1) core_sigma_cluster_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, int b, double* __restrict__ sigma,
    int* __restrict__ status) {
    constexpr int P2 = 2 * CL;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int nloc = (s + CL - 1) / CL;
    const int sp = (s + 31) / 32 * 32;                         // padded column length of R^T
    float* W = reinterpret_cast<float*>(smem);                // nloc x r2 (column-major)
    float* slot0 = W + (size_t)nloc * r2;                     // b columns of R^T (length s)
    float* slot1 = slot0 + (size_t)b * sp;
    float* vbuf = slot1 + (size_t)b * sp;                     // 2 x r2 Householder vectors
    __shared__ float s_tau[2];
    __shared__ int s_block[2];
    __shared__ int s_count, s_bad;
    __shared__ unsigned int s_meas;
    __shared__ float s_fmax;
    __shared__ unsigned long long s_dmax;
    __shared__ double s_norm[512];
    __shared__ float s_red[32];
    const int k = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    // ---- own columns: finiteness and the power-of-two scale agreed across the cluster
    if (tid == 0) {
        s_bad = 0;
        s_dmax = 0ull;
        s_count = 0;
        s_meas = 0u;
    }
    __syncthreads();
    {
        double mx = 0.0;
        int bad = 0;
        for (int64_t idx = tid; idx < (int64_t)nloc * r2; idx += blockDim.x) {
            const int jl = (int)(idx / r2), i = (int)(idx % r2);
            const int j = jl * CL + k;
            const double v = j < s ? core[(int64_t)i * ld + j] : 0.0;
            bad |= !isfinite(v);
            mx = fmax(mx, fabs(v));
        }
        if (bad) s_bad = 1;
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0 && isfinite(mx)) atomicMax(&s_dmax, (unsigned long long)__double_as_longlong(mx));
    }
    cluster.sync();
    int any_bad = 0;
    double gmax = 0.0;
    for (int r = 0; r < CL; ++r) {
        any_bad |= *cluster.map_shared_rank(&s_bad, r);
        gmax = fmax(gmax, __longlong_as_double((long long)*cluster.map_shared_rank(&s_dmax, r)));
    }
    if (any_bad) {
        if (k == 0) {
            for (int j = tid; j < s; j += blockDim.x) sigma[j] = nan("");
            if (tid == 0) *status = RE_ERR_NONFINITE;
        }
        cluster.sync();
        return;
    }
    int e2 = 0;
    if (gmax > 0.0) frexp(gmax, &e2);
    const double down = ldexp(1.0, -e2), up = ldexp(1.0, e2);
    for (int64_t idx = tid; idx < (int64_t)nloc * r2; idx += blockDim.x) {
        const int jl = (int)(idx / r2), i = (int)(idx % r2);
        const int j = jl * CL + k;
        W[idx] = j < s ? (float)(core[(int64_t)i * ld + j] * down) : 0.f;
    }
    cluster.sync();   // all CTAs have read every s_bad / s_dmax

    // ---- column-cyclic Householder QR
    for (int kk = 0; kk < s; ++kk) {
        const int owner = kk % CL, jl = kk / CL, buf = kk & 1;
        const int L = r2 - kk;
        if (k == owner) {
            float* colk = W + (size_t)jl * r2 + kk;
            if (warp == 0) {
                const float tau = householder(colk, L);
                if (lane == 0) s_tau[buf] = tau;
            }
            __syncthreads();
            const float tau = s_tau[buf];
            for (int r = 0; r < CL; ++r) {      // push v (leading 1) and tau to every CTA
                float* dst = cluster.map_shared_rank(vbuf + (size_t)buf * r2, r);
                for (int i = tid; i < L; i += blockDim.x) dst[i] = i == 0 ? 1.f : colk[i];
                if (tid == 0) *cluster.map_shared_rank(&s_tau[buf], r) = tau;
            }
        }
        cluster.sync();
        const float tau = s_tau[buf];
        const float* v = vbuf + (size_t)buf * r2;
        if (tau != 0.f) {
            const int first = (kk + 1 - k + CL - 1) / CL;     // smallest jl with jl*CL + k > kk
            for (int j2 = first + warp; j2 < nloc; j2 += nwarps) {
                float* cj = W + (size_t)j2 * r2 + kk;
                float w = 0.f;
                for (int i = lane; i < L; i += 32) w = fmaf(v[i], cj[i], w);
                w = warp_sum(w) * tau;
                for (int i = lane; i < L; i += 32) cj[i] = fmaf(-w, v[i], cj[i]);
            }
        }
        __syncthreads();
    }
    cluster.sync();

    // ---- gather the two R^T column blocks of this CTA (positions k and P2-1-k)
    if (tid == 0) {
        s_block[0] = k;
        s_block[1] = P2 - 1 - k;
    }
    for (int64_t idx = tid; idx < 2 * (int64_t)b * sp; idx += blockDim.x) {
        const int sl = (int)(idx / ((int64_t)b * sp));
        const int64_t off = idx % ((int64_t)b * sp);
        const int jj = (int)(off / sp), col = (int)(off % sp);   // entry col of R^T column c
        const int blk = sl == 0 ? k : P2 - 1 - k;
        const int c = blk * b + jj;                              // = row c of R
        float val = 0.f;
        if (c < s && col >= c && col < s) {
            const float* src = cluster.map_shared_rank(W, col % CL);
            val = src[(size_t)(col / CL) * r2 + c];
        }
        slot0[idx] = val;                                        // slot1 follows slot0
    }
    cluster.sync();

    // ---- blocked Jacobi on R^T (length-s columns)
    const float tol = 4.f * kU * sqrtf((float)s);
    float stage[kPullRegs];
    const int per_thread = (2 * b * sp + kSvdThreads - 1) / kSvdThreads;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        float amax = 0.f;
        for (int q = warp; q < 2 * b; q += nwarps) {
            const float* a = slot0 + (size_t)q * sp;
            float acc = 0.f;
            for (int i = lane; i < sp; i += 32) acc = fmaf(a[i], a[i], acc);
            amax = fmaxf(amax, warp_sum(acc));
        }
        if (lane == 0) s_red[warp] = amax;
        __syncthreads();
        if (warp == 0) {
            const float vv = warp_max(lane < nwarps ? s_red[lane] : 0.f);
            if (lane == 0) s_fmax = vv;
        }
        cluster.sync();
        float gm = 0.f;
        for (int r = 0; r < CL; ++r) gm = fmaxf(gm, *cluster.map_shared_rank(&s_fmax, r));
        const float floor_abs = kAbsFloor * gm;
        for (int t = 0; t < P2 - 1; ++t) {
            int rotated = 0;
            const int grp = tid / kG, ngrp = blockDim.x / kG;
            const bool leader = (tid & (kG - 1)) == 0;
            if (t == 0) {
                // pairs inside each block (circle ordering on b columns)
                const int P = b + (b & 1);
                for (int u = 0; u < P - 1; ++u) {
                    for (int base = 0; base < P; base += ngrp) {
                        const int q = base + grp;
                        bool act = q < P;
                        float* pa = slot0;
                        float* pb = slot0;
                        if (act) {
                            const int sl = q / (P / 2), kq = q % (P / 2);
                            const int i1 = kq, i2 = P - 1 - kq;
                            const int c1 = (i1 == 0) ? 0 : 1 + (i1 - 1 + u) % (P - 1);
                            const int c2 = (i2 == 0) ? 0 : 1 + (i2 - 1 + u) % (P - 1);
                            const int p = min(c1, c2), qq = max(c1, c2);
                            act = qq < b;
                            float* bs = sl == 0 ? slot0 : slot1;
                            pa = bs + (size_t)p * sp;
                            pb = bs + (size_t)qq * sp;
                        }
                        float meas = 0.f;
                        if (rotate_pair(act, pa, pb, sp, tol, floor_abs, &meas) && leader) {
                            rotated = 1;
                            atomicMax(&s_meas, __float_as_uint(meas));
                        }
                    }
                    __syncthreads();
                }
            }
            // cross pairs: in inner round u, column j of slot 0 meets column (j+u) mod b of slot 1
            for (int u = 0; u < b; ++u) {
                for (int base = 0; base < b; base += ngrp) {
                    const int j = base + grp;
                    const bool act = j < b;
                    const int jj = act ? (j + u) % b : 0;
                    float meas = 0.f;
                    if (rotate_pair(act, slot0 + (size_t)(act ? j : 0) * sp, slot1 + (size_t)jj * sp, sp, tol,
                                    floor_abs, &meas) && leader) {
                        rotated = 1;
                        atomicMax(&s_meas, __float_as_uint(meas));
                    }
                }
                __syncthreads();
            }
            if (rotated) atomicAdd(&s_count, 1);
            // tournament positions 1..P2-1 move up by one; pull the new blocks
            cluster.sync();
            const int src0 = (k == 0) ? -1 : (k == 1 ? P2 - 1 : k - 1);
            const int src1 = P2 - 2 - k;
            auto cta_of = [](int pos) { return pos < CL ? pos : P2 - 1 - pos; };
            auto slot_of = [](int pos) { return pos < CL ? 0 : 1; };
            int nb0 = s_block[0];
            const int nb1 = cluster.map_shared_rank(&s_block[0], cta_of(src1))[slot_of(src1)];
            if (src0 >= 0) nb0 = cluster.map_shared_rank(&s_block[0], cta_of(src0))[slot_of(src0)];
#pragma unroll
            for (int q = 0; q < kPullRegs; ++q) {
                const int64_t idx = (int64_t)q * kSvdThreads + tid;
                if (q < per_thread && idx < 2 * (int64_t)b * sp) {
                    const int sl = (int)(idx / ((int64_t)b * sp));
                    const int64_t off = idx % ((int64_t)b * sp);
                    const int src = sl == 0 ? src0 : src1;
                    if (src >= 0) {
                        const float* rs = cluster.map_shared_rank(slot0, cta_of(src));
                        stage[q] = rs[(size_t)slot_of(src) * b * sp + off];
                    } else {
                        stage[q] = slot0[off];
                    }
                }
            }
            cluster.sync();
#pragma unroll
            for (int q = 0; q < kPullRegs; ++q) {
                const int64_t idx = (int64_t)q * kSvdThreads + tid;
                if (q < per_thread && idx < 2 * (int64_t)b * sp) slot0[idx] = stage[q];
            }
            if (tid == 0) {
                s_block[0] = nb0;
                s_block[1] = nb1;
            }
            __syncthreads();
        }
        cluster.sync();
        int total = 0;
        float worst = 0.f;
        for (int r = 0; r < CL; ++r) {
            total += *cluster.map_shared_rank(&s_count, r);
            worst = fmaxf(worst, __uint_as_float(*cluster.map_shared_rank(&s_meas, r)));
        }
        cluster.sync();
        if (tid == 0) {
            s_count = 0;
            s_meas = 0u;
        }
        __syncthreads();
        if (k == 0 && tid == 0) status[2] = sweep + 1;
        if (total == 0 || worst < kStopFactor * kU * sqrtf((float)s)) break;
    }
    // ---- norms gathered in CTA 0
    for (int q = warp; q < 2 * b; q += nwarps) {
        const int sl = q / b, j = q % b;
        const int c = s_block[sl] * b + j;
        const double nv = col_norm(slot0 + (size_t)q * sp, sp);
        if (lane == 0 && c < s) *cluster.map_shared_rank(&s_norm[c], 0) = nv;
    }
    cluster.sync();
    if (k == 0) {
        sort_desc(s_norm, s, up, sigma);
        if (tid == 0) *status = RE_OK;
    }
}

size_t cluster_smem(int CL, int r2, int s, int* b_out) {
    const int nloc = (s + CL - 1) / CL;
    const int b = (s + 2 * CL - 1) / (2 * CL);
    const size_t sp = (size_t)(s + 31) / 32 * 32;
    *b_out = b;
    return sizeof(float) * ((size_t)nloc * r2 + 2 * (size_t)b * sp + 2 * (size_t)r2);
}

template <int CL>
cudaError_t launch_cluster_sigma(const double* core, int r2, int s, int64_t ld, double* sigma,
                                 int* status, cudaStream_t st) {
    int b = 0;
    const size_t smem = cluster_smem(CL, r2, s, &b);
    if (2 * (size_t)b * ((s + 31) / 32 * 32) > (size_t)kPullRegs * kSvdThreads) return cudaErrorInvalidValue;
    auto kern = core_sigma_cluster_kernel<CL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (CL > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(kSvdThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, core, r2, s, ld, b, sigma, status);
}

// Step 8 (device): scaled sigma, threshold rank, gap index.
__global__ void readoff_kernel(const double* __restrict__ sigma, int r1, double scale, double eps,
                               double norm_a, const int* __restrict__ status_in,
                               DevReadoff* __restrict__ out, double* __restrict__ sigma_scaled) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevReadoff r;
    // status_in[0]: small-core step (RE_OK / RE_ERR_NONFINITE); status_in[1]: set
    // by the tensor-core right sketch when one of its bounded waits expired
    r.status = status_in ? status_in[0] : RE_OK;
    if (status_in && status_in[1]) r.status = RE_ERR_TIMEOUT;
    r.sweeps = status_in ? status_in[2] : 0;
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

constexpr size_t kSmemLimit = 210 * 1024;

size_t cta_smem(int r2, int s) {
    const size_t sp = (size_t)(s + 31) / 32 * 32;
    return sizeof(float) * ((size_t)r2 * s + sp * s);
}

}  // namespace

size_t svd_workspace_bytes(int, int) { return 256; }

bool core_sigma_fits_cta(int r2, int s) { return cta_smem(r2, s) <= kSmemLimit; }

cudaError_t launch_core_sigma_batched(const double* core, int r2, int s, int64_t ld,
                                      int64_t core_stride, int count, double* sigma,
                                      int64_t sigma_stride, int* status, cudaStream_t st) {
    const size_t sm = cta_smem(r2, s);
    if (sm > kSmemLimit || count <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(core_sigma_cta_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    core_sigma_cta_kernel<<<count, kSvdThreads, sm, st>>>(core, r2, s, ld, core_stride, sigma,
                                                          sigma_stride, status);
    return cudaGetLastError();
}

cudaError_t launch_core_sigma(const double* core, int r2, int s, int64_t ld, void*, double* sigma,
                              int* status, cudaStream_t st) {
    if (s <= 0) return cudaSuccess;
    if (s > 512) return cudaErrorInvalidValue;
    if (cta_smem(r2, s) <= kSmemLimit)
        return launch_core_sigma_batched(core, r2, s, ld, 0, 1, sigma, 0, status, st);
    int b = 0;
    const size_t sp = (size_t)(s + 31) / 32 * 32;
    if (cluster_smem(8, r2, s, &b) <= kSmemLimit && 2 * (size_t)b * sp <= (size_t)kPullRegs * kSvdThreads)
        return launch_cluster_sigma<8>(core, r2, s, ld, sigma, status, st);
    if (cluster_smem(16, r2, s, &b) <= kSmemLimit && 2 * (size_t)b * sp <= (size_t)kPullRegs * kSvdThreads)
        return launch_cluster_sigma<16>(core, r2, s, ld, sigma, status, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_readoff(const double* sigma, int r1, double scale, double eps, double norm_a,
                           const int* status_in, DevReadoff* out, double* sigma_scaled,
                           cudaStream_t st) {
    readoff_kernel<<<1, 32, 0, st>>>(sigma, r1, scale, eps, norm_a, status_in, out, sigma_scaled);
    return cudaGetLastError();
}

}  // namespace re
