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
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cmath>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

namespace cg = cooperative_groups;

constexpr int kSvdThreads = 512;      // cluster kernel
constexpr int kCtaThreads = 1024;     // one-CTA kernel: 64 column pairs x 16 lanes
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

// Jacobi rotation of columns a, b (length 4*G*NV, 16-byte aligned) by a group
// of G consecutive lanes; each lane holds NV float4 of each column in registers
// (elements 4 (gl + G v) .. +3), so the columns are read once and written once.
// Every lane of the warp must call it (the reductions use full-warp shuffles);
// inactive groups pass active = false.  A pair is rotated when
// |a.b| > tol |a| |b| and |a.b| > floor_abs; then rotated is set and meas_max
// takes max(|cos|).  The rotation parameters use the fast reciprocal square
// root and division: their rounding only perturbs the angle, and c^2 + s^2
// stays 1 to a few ulp.
template <int G, int NV>
__device__ __forceinline__ void jacobi_pair(bool active, float* a, float* b, float tol2, float floor_abs,
                                            float& meas_max, int& rotated) {
    const int gl = threadIdx.x & (G - 1);
    float4 x[NV], y[NV];
    float al = 0.f, be = 0.f, ga = 0.f, al2 = 0.f, be2 = 0.f, ga2 = 0.f;
    if (active) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            x[v] = *reinterpret_cast<const float4*>(a + 4 * (gl + G * v));
            y[v] = *reinterpret_cast<const float4*>(b + 4 * (gl + G * v));
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            al = fmaf(x[v].x, x[v].x, fmaf(x[v].y, x[v].y, al));
            al2 = fmaf(x[v].z, x[v].z, fmaf(x[v].w, x[v].w, al2));
            be = fmaf(y[v].x, y[v].x, fmaf(y[v].y, y[v].y, be));
            be2 = fmaf(y[v].z, y[v].z, fmaf(y[v].w, y[v].w, be2));
            ga = fmaf(x[v].x, y[v].x, fmaf(x[v].y, y[v].y, ga));
            ga2 = fmaf(x[v].z, y[v].z, fmaf(x[v].w, y[v].w, ga2));
        }
    }
    al += al2;
    be += be2;
    ga += ga2;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
    }
    const float ag = fabsf(ga);
    const float ab = al * be;
    // ga^2 > tol^2 al be  <=>  |ga| > tol |a| |b|  (pairs below the absolute floor are
    // skipped first, so al be cannot have underflowed for a rotated pair)
    if (!active || !(ag > floor_abs) || !(ga * ga > tol2 * ab)) return;
    rotated = 1;
    meas_max = fmaxf(meas_max, ag * rsqrtf(ab));
    const float zeta = __fdividef(be - al, ga + ga);
    const float az = fabsf(zeta);
    float tt;
    if (az > 1e15f) {
        tt = __fdividef(0.5f, zeta);
    } else {
        const float q = fmaf(zeta, zeta, 1.f);
        tt = copysignf(__fdividef(1.f, az + q * rsqrtf(q)), zeta);
    }
    const float c = rsqrtf(fmaf(tt, tt, 1.f));
    const float sn = c * tt;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const float4 xa = x[v], ya = y[v];
        x[v].x = fmaf(c, xa.x, -sn * ya.x);
        x[v].y = fmaf(c, xa.y, -sn * ya.y);
        x[v].z = fmaf(c, xa.z, -sn * ya.z);
        x[v].w = fmaf(c, xa.w, -sn * ya.w);
        y[v].x = fmaf(sn, xa.x, c * ya.x);
        y[v].y = fmaf(sn, xa.y, c * ya.y);
        y[v].z = fmaf(sn, xa.z, c * ya.z);
        y[v].w = fmaf(sn, xa.w, c * ya.w);
        *reinterpret_cast<float4*>(a + 4 * (gl + G * v)) = x[v];
        *reinterpret_cast<float4*>(b + 4 * (gl + G * v)) = y[v];
    }
}

// Warp-wide OR of `rotated` and max of `meas` folded into shared flags (one
// atomic per warp).
__device__ __forceinline__ void fold_sweep_flags(int rotated, float meas, int* s_any, unsigned int* s_meas) {
    const int any = __any_sync(0xffffffffu, rotated);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) meas = fmaxf(meas, __shfl_xor_sync(0xffffffffu, meas, o));
    if ((threadIdx.x & 31) == 0 && any) {
        atomicOr(s_any, 1);
        atomicMax(s_meas, __float_as_uint(meas));
    }
}

// Position i of the round-robin (circle) schedule on P players in round t.
__device__ __forceinline__ int circle_player(int i, int t, int P) {
    if (i == 0) return 0;
    int x = i - 1 + t;
    if (x >= P - 1) x -= P - 1;
    return 1 + x;
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

// Register-resident versions for a column of length L <= 32*E (one warp; lane
// l holds entries l, l+32, ..., masked past L).  householder_regs: reflector of
// x = col[0..L) with the same arithmetic as householder(); v (v[0] = 1) goes to
// col[1..), beta to col[0]; returns tau.
template <int E>
__device__ __forceinline__ float householder_regs(float* col, int L) {
    const int lane = threadIdx.x & 31;
    float x[E];
    float ss = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        x[e] = i < L ? col[i] : 0.f;
        if (i >= 1) ss = fmaf(x[e], x[e], ss);
    }
    ss = warp_sum(ss);
    const float x0 = __shfl_sync(0xffffffffu, x[0], 0);
    float tau = 0.f, beta = x0;
    if (ss > 0.f) {
        const float nrm = sqrtf(fmaf(x0, x0, ss));
        beta = -copysignf(nrm, x0);
        tau = (beta - x0) / beta;
        const float scale = 1.f / (x0 - beta);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane + 32 * e;
            if (i >= 1 && i < L) col[i] = x[e] * scale;
        }
    }
    if (lane == 0) col[0] = beta;
    __syncwarp();
    return tau;
}

// Load v (v[0] = 1, entries 1..L-1 from vsrc) into registers.
template <int E>
__device__ __forceinline__ void load_reflector(const float* vsrc, int L, float (&v)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        v[e] = i < L ? (i == 0 ? 1.f : vsrc[i]) : 0.f;
    }
}

// c <- (I - tau v v^T) c for one column of length L (one warp).
template <int E>
__device__ __forceinline__ void apply_reflector(const float (&v)[E], float tau, float* c, int L) {
    const int lane = threadIdx.x & 31;
    float x[E];
    float w = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        x[e] = i < L ? c[i] : 0.f;
        w = fmaf(v[e], x[e], w);
    }
    w = warp_sum(w) * tau;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < L) c[i] = fmaf(-w, v[e], x[e]);
    }
}

// ---------------------------------------------------------------------------
// One CTA per core: core -> shared memory (column-major, scaled), QR in place,
// R^T -> second region, Jacobi on R^T, norms.  blockIdx.x selects the core
// (core_stride / sigma_stride apart) so one launch serves a batch.
template <int NV, int E>
__global__ void __launch_bounds__(kCtaThreads, 1) core_sigma_cta_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, int64_t core_stride,
    double* __restrict__ sigma, int64_t sigma_stride, int* __restrict__ status,
    const int* __restrict__ active, int cert_r1, float cert_ratio) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (active && !active[blockIdx.x]) return;
    core += (int64_t)blockIdx.x * core_stride;
    sigma += (int64_t)blockIdx.x * sigma_stride;
    const int sp = 64 * NV;                             // padded column length of R^T (4 x 16 lanes x NV)
    float* W = reinterpret_cast<float*>(smem);          // r2 x s, column-major
    float* Rt = W + ((size_t)r2 * s + 31) / 32 * 32;    // sp x s, column c = row c of R (128-B aligned)
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

    // Householder QR: column k's reflector, then the trailing columns (reflector
    // and each column held in registers, r2 <= 32 E)
    for (int k = 0; k < s; ++k) {
        float* colk = W + (size_t)k * r2 + k;
        const int L = r2 - k;
        if (warp == 0) {
            const float tau = householder_regs<E>(colk, L);
            if (lane == 0) s_tau = tau;
        }
        __syncthreads();
        const float tau = s_tau;
        if (tau != 0.f && k + 1 + warp < s) {
            float v[E];
            load_reflector<E>(colk, L, v);
            for (int j = k + 1 + warp; j < s; j += nwarps) apply_reflector<E>(v, tau, W + (size_t)j * r2 + k, L);
        }
        __syncthreads();
    }
    // Certificate of non-convergence (used at intermediate ladder widths only):
    // sigma_r1(core) >= sigma_min(R11) >= 1 / ||R11^{-1}||_F (column interlacing)
    // and sigma_1(core) <= ||R||_F; when the lower bound exceeds cert_ratio times
    // the upper bound, the read-off cannot succeed at this width and the Jacobi
    // sweeps are skipped (status[3] = 1; sigma is not written).
    if (cert_r1 > 0 && cert_r1 <= s) {
        __shared__ float s_fro, s_inv;
        __shared__ int s_zero;
        if (tid == 0) {
            s_fro = 0.f;
            s_inv = 0.f;
            s_zero = 0;
        }
        __syncthreads();
        float fro = 0.f;
        for (int64_t idx = tid; idx < (int64_t)s * s; idx += blockDim.x) {
            const int j = (int)(idx / s), i = (int)(idx % s);
            if (i <= j) {
                const float v = W[(size_t)j * r2 + i];
                fro = fmaf(v, v, fro);
            }
        }
        fro = warp_sum(fro);
        if (lane == 0) atomicAdd(&s_fro, fro);
        // columns of R11^{-1} by back substitution, one warp per column
        float* x = Rt + (size_t)warp * sp;             // Rt is free until the transpose below
        float inv = 0.f;
        for (int j = warp; j < cert_r1; j += nwarps) {
            const float rjj = W[(size_t)j * r2 + j];
            if (rjj == 0.f) {
                if (lane == 0) s_zero = 1;
                continue;
            }
            if (lane == 0) x[j] = 1.f / rjj;
            __syncwarp();
            float acc = lane == 0 ? x[j] * x[j] : 0.f;
            for (int i = j - 1; i >= 0; --i) {
                float t = 0.f;
                for (int k = i + 1 + lane; k <= j; k += 32) t = fmaf(W[(size_t)k * r2 + i], x[k], t);
                t = warp_sum(t);
                const float rii = W[(size_t)i * r2 + i];
                const float xi = rii != 0.f ? -t / rii : INFINITY;
                if (lane == 0) {
                    x[i] = xi;
                    acc = fmaf(xi, xi, acc);
                }
                __syncwarp();
            }
            inv += acc;
        }
        if (lane == 0) atomicAdd(&s_inv, inv);
        __syncthreads();
        const bool certified = s_zero == 0 && isfinite(s_inv) && s_inv > 0.f &&
                               1.f / sqrtf(s_inv) > cert_ratio * sqrtf(s_fro);
        __syncthreads();
        if (certified) {
            if (tid == 0 && sigma_stride == 0) status[3] = 1;
            if (tid == 0) status[blockIdx.x] = RE_OK;
            return;
        }
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
        constexpr int G = 16;
        const int grp = tid / G, ngrp = blockDim.x / G;
        int rotated = 0;
        float meas = 0.f;
        for (int t = 0; t < P - 1; ++t) {
            for (int base = 0; base < P / 2; base += ngrp) {
                const int q = base + grp;
                int p = 0, qq = 0;
                bool act = q < P / 2;
                if (act) {
                    const int c1 = circle_player(q, t, P), c2 = circle_player(P - 1 - q, t, P);
                    p = min(c1, c2);
                    qq = max(c1, c2);
                    act = qq < s;
                }
                jacobi_pair<G, NV>(act, Rt + (size_t)p * sp, Rt + (size_t)qq * sp, tol * tol, floor_abs, meas,
                                   rotated);
            }
            __syncthreads();
        }
        fold_sweep_flags(rotated, meas, &s_flag, &s_meas);
        __syncthreads();
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

template <int CL, int NV, int E>
__global__ void __launch_bounds__(kSvdThreads, 1) core_sigma_cluster_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, int b, double* __restrict__ sigma,
    int* __restrict__ status) {
    constexpr int P2 = 2 * CL;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int nloc = (s + CL - 1) / CL;
    const int sp = 128 * NV;                                   // padded column length of R^T
    const size_t set_floats = 2 * (size_t)b * sp;              // two blocks of b columns
    const size_t r1_floats = (max((size_t)nloc * r2, set_floats) + 31) / 32 * 32;
    float* W = reinterpret_cast<float*>(smem);                // QR: nloc x r2 (column-major)
    float* vbuf = W + r1_floats;                              // 2 x r2 Householder vectors
    float* sets[2] = {vbuf + (2 * (size_t)r2 + 31) / 32 * 32, W};   // Jacobi ping-pong (set 1 reuses W)
    __shared__ float s_tau[2];
    __shared__ int s_block[2][2];                             // [set][slot] block ids
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
                const float tau = householder_regs<E>(colk, L);
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
        const int first = (kk + 1 - k + CL - 1) / CL;         // smallest jl with jl*CL + k > kk
        if (tau != 0.f && first + warp < nloc) {
            float vr[E];
            load_reflector<E>(v, L, vr);
            for (int j2 = first + warp; j2 < nloc; j2 += nwarps)
                apply_reflector<E>(vr, tau, W + (size_t)j2 * r2 + kk, L);
        }
        __syncthreads();
    }
    cluster.sync();

    // ---- gather the two R^T column blocks of this CTA (positions k and P2-1-k)
    if (tid == 0) {
        s_block[0][0] = k;
        s_block[0][1] = P2 - 1 - k;
    }
    float* slot0 = sets[0];
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

    // ---- blocked Jacobi on R^T (length-sp columns, zero padded)
    const float tol = 4.f * kU * sqrtf((float)s);
    int cur = 0;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        float amax = 0.f;
        for (int q = warp; q < 2 * b; q += nwarps) {
            const float* a = sets[cur] + (size_t)q * sp;
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
        int rotated = 0;
        float meas = 0.f;
        for (int t = 0; t < P2 - 1; ++t) {
            float* c0 = sets[cur];
            float* c1 = c0 + (size_t)b * sp;
            constexpr int G = 32;                  // one warp per pair: few pairs per round
            const int grp = tid / G, ngrp = blockDim.x / G;
            if (t == 0) {
                // pairs inside each block (circle ordering on b columns)
                const int P = b + (b & 1);
                for (int u = 0; u < P - 1; ++u) {
                    for (int base = 0; base < P; base += ngrp) {
                        const int q = base + grp;
                        bool act = q < P;
                        float* pa = c0;
                        float* pb = c0;
                        if (act) {
                            const int sl = q / (P / 2), kq = q % (P / 2);
                            const int e1 = circle_player(kq, u, P), e2 = circle_player(P - 1 - kq, u, P);
                            const int p = min(e1, e2), qq = max(e1, e2);
                            act = qq < b;
                            float* bs = sl == 0 ? c0 : c1;
                            pa = bs + (size_t)p * sp;
                            pb = bs + (size_t)qq * sp;
                        }
                        jacobi_pair<G, NV>(act, pa, pb, tol * tol, floor_abs, meas, rotated);
                    }
                    __syncthreads();
                }
            }
            // cross pairs: in inner round u, column j of slot 0 meets column (j+u) mod b of slot 1
            for (int u = 0; u < b; ++u) {
                for (int base = 0; base < b; base += ngrp) {
                    const int j = base + grp;
                    const bool act = j < b;
                    int jj = act ? j + u : 0;
                    if (jj >= b) jj -= b;
                    jacobi_pair<G, NV>(act, c0 + (size_t)(act ? j : 0) * sp, c1 + (size_t)jj * sp, tol * tol,
                                       floor_abs, meas, rotated);
                }
                __syncthreads();
            }
            // tournament positions 1..P2-1 move up by one: pull the new blocks from
            // the current set of their source CTAs into this CTA's other set
            cluster.sync();
            const int src0 = (k == 0) ? -1 : (k == 1 ? P2 - 1 : k - 1);
            const int src1 = P2 - 2 - k;
            auto cta_of = [](int pos) { return pos < CL ? pos : P2 - 1 - pos; };
            auto slot_of = [](int pos) { return pos < CL ? 0 : 1; };
            const int nxt = cur ^ 1;
            const int n4 = b * sp / 4;
            for (int sl = 0; sl < 2; ++sl) {
                const int src = sl == 0 ? src0 : src1;
                const float4* from;
                if (src >= 0) {
                    const float* rs = cluster.map_shared_rank(sets[cur], cta_of(src));
                    from = reinterpret_cast<const float4*>(rs + (size_t)slot_of(src) * b * sp);
                } else {
                    from = reinterpret_cast<const float4*>(sets[cur]);
                }
                float4* to = reinterpret_cast<float4*>(sets[nxt] + (size_t)sl * b * sp);
                for (int i = tid; i < n4; i += blockDim.x) to[i] = from[i];
            }
            if (tid == 0) {
                s_block[nxt][0] = src0 >= 0
                                      ? cluster.map_shared_rank(&s_block[cur][0], cta_of(src0))[slot_of(src0)]
                                      : s_block[cur][0];
                s_block[nxt][1] = cluster.map_shared_rank(&s_block[cur][0], cta_of(src1))[slot_of(src1)];
            }
            cur = nxt;
            __syncthreads();
        }
        fold_sweep_flags(rotated, meas, &s_count, &s_meas);
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
    slot0 = sets[cur];
    // ---- norms gathered in CTA 0
    for (int q = warp; q < 2 * b; q += nwarps) {
        const int sl = q / b, j = q % b;
        const int c = s_block[cur][sl] * b + j;
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
    const size_t sp = (size_t)(s + 127) / 128 * 128;
    const size_t set_floats = 2 * (size_t)b * sp;
    *b_out = b;
    return sizeof(float) * ((std::max((size_t)nloc * r2, set_floats) + 31) / 32 * 32 +
                            (2 * (size_t)r2 + 31) / 32 * 32 + set_floats);
}

template <int CL, int NV, int E>
cudaError_t launch_cluster_sigma_nv(const double* core, int r2, int s, int64_t ld, double* sigma,
                                    int* status, cudaStream_t st) {
    int b = 0;
    const size_t smem = cluster_smem(CL, r2, s, &b);
    auto kern = core_sigma_cluster_kernel<CL, NV, E>;
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

template <int CL, int NV>
cudaError_t launch_cluster_sigma_e(const double* core, int r2, int s, int64_t ld, double* sigma, int* status,
                                   cudaStream_t st) {
    // column length r2 <= 32 E; this kernel only takes cores that do not fit one CTA (r2 > 128)
    const int e = (r2 + 31) / 32;
    if (e <= 8) return launch_cluster_sigma_nv<CL, NV, 8>(core, r2, s, ld, sigma, status, st);
    if (e <= 16) return launch_cluster_sigma_nv<CL, NV, 16>(core, r2, s, ld, sigma, status, st);
    if (e <= 32) return launch_cluster_sigma_nv<CL, NV, 32>(core, r2, s, ld, sigma, status, st);
    return cudaErrorInvalidValue;
}

template <int CL>
cudaError_t launch_cluster_sigma(const double* core, int r2, int s, int64_t ld, double* sigma,
                                 int* status, cudaStream_t st) {
    switch ((s + 127) / 128) {
        case 1: return launch_cluster_sigma_e<CL, 1>(core, r2, s, ld, sigma, status, st);
        case 2: return launch_cluster_sigma_e<CL, 2>(core, r2, s, ld, sigma, status, st);
        case 3: return launch_cluster_sigma_e<CL, 3>(core, r2, s, ld, sigma, status, st);
        case 4: return launch_cluster_sigma_e<CL, 4>(core, r2, s, ld, sigma, status, st);
        default: return cudaErrorInvalidValue;
    }
}

// Step 8 (device): scaled sigma, threshold rank, gap index.
// One warp: lanes take indices i = lane, lane + 32, ...; the threshold rank is the
// smallest index with sigma^ <= tau and the gap the largest ratio, smallest index on
// ties (the same values and decisions as a sequential scan).
__global__ void readoff_kernel(const double* __restrict__ sigma, int r1, double scale, double eps,
                               double norm_a, const int* __restrict__ status_in,
                               DevReadoff* __restrict__ out, double* __restrict__ sigma_scaled) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    DevReadoff r;
    // status_in[0]: small-core step (RE_OK / RE_ERR_NONFINITE); status_in[1]: set
    // by a tensor-core kernel when one of its bounded waits expired
    r.status = status_in ? status_in[0] : RE_OK;
    if (status_in && status_in[1]) r.status = RE_ERR_TIMEOUT;
    if (status_in && status_in[3]) {
        // the core step certified that no trusted sigma^ reaches the threshold
        if (lane == 0) {
            r.sweeps = 0;
            r.rank = -1;
            r.gap_index = 0;
            r.gap_ratio = 0.0;
            r.tau = 0.0;
            *out = r;
        }
        return;
    }
    r.sweeps = status_in ? status_in[2] : 0;
    const double ref = norm_a > 0.0 ? norm_a : sigma[0] * scale;
    r.tau = eps * ref;
    int first = INT_MAX;
    int gi = r1 >= 1 ? 1 : 0;
    double gr = r1 >= 2 ? -1.0 : 1.0;
    for (int i = lane; i < r1; i += 32) {
        const double v = sigma[i] * scale;
        sigma_scaled[i] = v;
        if (v <= r.tau && i < first) first = i;
        if (i >= 1) {
            const double a = sigma[i - 1] * scale;
            double ratio;
            if (v > 0.0) ratio = a / v;
            else if (a > 0.0) ratio = INFINITY;
            else ratio = 1.0;
            if (ratio > gr || (ratio == gr && i < gi)) {
                gr = ratio;
                gi = i;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        const double g2 = __shfl_xor_sync(0xffffffffu, gr, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, gi, o);
        if (g2 > gr || (g2 == gr && i2 < gi)) {
            gr = g2;
            gi = i2;
        }
    }
    if (lane == 0) {
        r.rank = first == INT_MAX ? -1 : first;
        r.gap_index = gi;
        r.gap_ratio = gr;
        *out = r;
    }
}

constexpr size_t kSmemLimit = 210 * 1024;

size_t cta_smem(int r2, int s) {
    const size_t sp = (size_t)(s + 63) / 64 * 64;
    return sizeof(float) * (((size_t)r2 * s + 31) / 32 * 32 + sp * s);
}

}  // namespace

size_t svd_workspace_bytes(int, int) { return 256; }

namespace {

using CtaKernel = void (*)(const double*, int, int, int64_t, int64_t, double*, int64_t, int*, const int*, int,
                           float);

template <int NV>
CtaKernel cta_kernel_e(int e) {
    if (e <= 1) return core_sigma_cta_kernel<NV, 1>;
    if (e <= 2) return core_sigma_cta_kernel<NV, 2>;
    if (e <= 4) return core_sigma_cta_kernel<NV, 4>;
    if (e <= 8) return core_sigma_cta_kernel<NV, 8>;
    if (e <= 16) return core_sigma_cta_kernel<NV, 16>;
    if (e <= 32) return core_sigma_cta_kernel<NV, 32>;
    return nullptr;
}

// instance for R^T column length 64 NV and core height r2 <= 32 e
CtaKernel cta_kernel_for(int nv, int e) {
    switch (nv) {
        case 1: return cta_kernel_e<1>(e);
        case 2: return cta_kernel_e<2>(e);
        case 3: return cta_kernel_e<3>(e);
        case 4: return cta_kernel_e<4>(e);
        default: return nullptr;
    }
}

}  // namespace

bool core_sigma_fits_cta(int r2, int s) { return cta_smem(r2, s) <= kSmemLimit; }

cudaError_t launch_core_sigma_batched(const double* core, int r2, int s, int64_t ld,
                                      int64_t core_stride, int count, double* sigma,
                                      int64_t sigma_stride, int* status, cudaStream_t st,
                                      const int* active, int cert_r1, float cert_ratio) {
    const size_t sm = cta_smem(r2, s);
    if (sm > kSmemLimit || count <= 0) return cudaErrorInvalidValue;
    auto kern = cta_kernel_for((s + 63) / 64, (r2 + 31) / 32);
    if (!kern) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<count, kCtaThreads, sm, st>>>(core, r2, s, ld, core_stride, sigma, sigma_stride, status, active,
                                         cert_r1, cert_ratio);
    return cudaGetLastError();
}

cudaError_t launch_core_sigma(const double* core, int r2, int s, int64_t ld, void*, double* sigma,
                              int* status, cudaStream_t st, int cert_r1, float cert_ratio) {
    if (s <= 0) return cudaSuccess;
    if (s > 512) return cudaErrorInvalidValue;
    if (cta_smem(r2, s) <= kSmemLimit)
        return launch_core_sigma_batched(core, r2, s, ld, 0, 1, sigma, 0, status, st, nullptr, cert_r1,
                                         cert_ratio);
    int b = 0;
    if (cluster_smem(8, r2, s, &b) <= kSmemLimit) return launch_cluster_sigma<8>(core, r2, s, ld, sigma, status, st);
    if (cluster_smem(16, r2, s, &b) <= kSmemLimit) return launch_cluster_sigma<16>(core, r2, s, ld, sigma, status, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_readoff(const double* sigma, int r1, double scale, double eps, double norm_a,
                           const int* status_in, DevReadoff* out, double* sigma_scaled,
                           cudaStream_t st) {
    readoff_kernel<<<1, 32, 0, st>>>(sigma, r1, scale, eps, norm_a, status_in, out, sigma_scaled);
    return cudaGetLastError();
}

}  // namespace re
