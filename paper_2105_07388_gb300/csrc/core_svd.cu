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
// and run on separate lane groups.
//
// Arithmetic is FP32: on GB300 FP64 runs at about 1/64 of the FP32 rate, and the
// sketch itself is accumulated in FP32, so FP32 rotations (absolute error about
// 1e-5 sigma_1 at s = 512) keep the whole path consistent.  Rotations whose
// off-diagonal term is below (1e-7 sigma_1)^2 are skipped: they cannot move any
// singular value by more than 1e-7 sigma_1, far below the FP32 noise floor.
// Rotations run two lanes of data per instruction (packed FP32x2 multiply and
// fused multiply-add, rounded per element exactly as the scalar forms).
//
// Small cores (r2 s + s^2 floats fit in shared memory) use one CTA; larger cores
// use two cluster kernels of 8 or 16 CTAs: a QR kernel (the columns dealt out in
// panels of 8; each panel factored on the CTA that owns it, which publishes its
// reflectors once through global memory, with one panel of lookahead: the owner
// of the next panel updates and factors it while the other CTAs update the
// rest), then a Jacobi kernel (two column blocks per CTA, blocks moving through
// the cluster each round).  Both QR forms factor panels of 8 columns with
// lookahead.
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

constexpr int kSvdThreads = 512;      // cluster QR kernel
constexpr int kJacThreads = 256;      // cluster Jacobi kernel
constexpr int kCtaThreads = 1024;     // one-CTA kernel: 64 column pairs x 16 lanes
constexpr int kMaxSweeps = 40;
constexpr int kPanel = 8;             // cluster QR: columns per panel
constexpr float kU = 5.9604644775390625e-08f;        // 2^-24
constexpr float kAbsFloor = 1e-14f;                  // (1e-7)^2 of max column norm^2
// A sweep whose largest rotated |cos| is below kStopFactor * u * sqrt(n) only
// rotated pairs at the FP32 rounding level of the dot products: stop there.
constexpr float kStopFactor = 32.f;
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

typedef unsigned long long u64;

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
__device__ __forceinline__ u64 warp_max(u64 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// |v| as its bit pattern: for finite doubles the unsigned order of these words is
// the order of |v|, and a word >= kInfBits marks Inf or NaN (integer work only:
// FP64 instructions issue at 1/64 rate on this part).
__device__ __forceinline__ u64 abs_bits(double v) {
    return (u64)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// packed FP32x2 (low word = first element)
__device__ __forceinline__ u64 pk2(float a, float b) {
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float sum2(u64 v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return a + b;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Jacobi rotation of two columns held in registers by a group of G consecutive
// lanes (each lane holds NV float4 of each column: elements 4 (gl + G v) .. +3).
// Every lane of the warp must call it (the reductions use full-warp shuffles);
// inactive groups pass active = false.  A pair is rotated when
// |a.b| > tol |a| |b| and |a.b| > floor_abs; then rotated is set, meas_max takes
// max(|cos|) and the function returns true.  The rotation parameters use the fast
// reciprocal square root and division: their rounding only perturbs the angle,
// and c^2 + s^2 stays 1 to a few ulp.  The dot products and the update run as
// packed FP32x2 instructions; each element is rounded as by the scalar fmaf /
// multiply.
template <int G, int NV>
__device__ __forceinline__ bool rotate_pair(bool active, ulonglong2 (&x)[NV], ulonglong2 (&y)[NV], float tol2,
                                            float floor_abs, float& meas_max, int& rotated) {
    u64 al0 = 0ull, al1 = 0ull, be0 = 0ull, be1 = 0ull, ga0 = 0ull, ga1 = 0ull;
    if (active) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            al0 = fma2(x[v].x, x[v].x, al0);
            al1 = fma2(x[v].y, x[v].y, al1);
            be0 = fma2(y[v].x, y[v].x, be0);
            be1 = fma2(y[v].y, y[v].y, be1);
            ga0 = fma2(x[v].x, y[v].x, ga0);
            ga1 = fma2(x[v].y, y[v].y, ga1);
        }
    }
    float al = sum2(add2(al0, al1));
    float be = sum2(add2(be0, be1));
    float ga = sum2(add2(ga0, ga1));
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
    if (!active || !(ag > floor_abs) || !(ga * ga > tol2 * ab)) return false;
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
    const u64 c2 = pk2(c, c), s2 = pk2(sn, sn), n2 = pk2(-sn, -sn);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const ulonglong2 xa = x[v], ya = y[v];
        x[v].x = fma2(c2, xa.x, mul2(n2, ya.x));     // c a - s b
        x[v].y = fma2(c2, xa.y, mul2(n2, ya.y));
        y[v].x = fma2(s2, xa.x, mul2(c2, ya.x));     // s a + c b
        y[v].y = fma2(s2, xa.y, mul2(c2, ya.y));
    }
    return true;
}

// rotate_pair on columns a, b in shared memory (length 4*G*NV, 16-byte aligned):
// each is read once and, when rotated, written once
template <int G, int NV>
__device__ __forceinline__ void jacobi_pair(bool active, float* a, float* b, float tol2, float floor_abs,
                                            float& meas_max, int& rotated) {
    const int gl = threadIdx.x & (G - 1);
    ulonglong2 x[NV], y[NV];
    if (active) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            x[v] = *reinterpret_cast<const ulonglong2*>(a + 4 * (gl + G * v));
            y[v] = *reinterpret_cast<const ulonglong2*>(b + 4 * (gl + G * v));
        }
    }
    if (rotate_pair<G, NV>(active, x, y, tol2, floor_abs, meas_max, rotated)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            *reinterpret_cast<ulonglong2*>(a + 4 * (gl + G * v)) = x[v];
            *reinterpret_cast<ulonglong2*>(b + 4 * (gl + G * v)) = y[v];
        }
    }
}

// rotate_pair of a register-held column x with column b in shared memory
template <int G, int NV>
__device__ __forceinline__ void jacobi_pair_x(bool active, ulonglong2 (&x)[NV], float* b, float tol2,
                                              float floor_abs, float& meas_max, int& rotated) {
    const int gl = threadIdx.x & (G - 1);
    ulonglong2 y[NV];
    if (active) {
#pragma unroll
        for (int v = 0; v < NV; ++v) y[v] = *reinterpret_cast<const ulonglong2*>(b + 4 * (gl + G * v));
    }
    if (rotate_pair<G, NV>(active, x, y, tol2, floor_abs, meas_max, rotated)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) *reinterpret_cast<ulonglong2*>(b + 4 * (gl + G * v)) = y[v];
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

// Descending rank sort of the non-negative s_norm[0..n) into out (scaled by
// `scale`); compares the bit patterns as integers (same order for x >= 0).
__device__ void sort_desc(const double* s_norm, int n, double scale, double* out) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double v = s_norm[j];
        const long long vb = __double_as_longlong(v);
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            const long long w = __double_as_longlong(s_norm[i]);
            rank += (w > vb) || (w == vb && i < j);
        }
        out[rank] = v * scale;
    }
}

// Column held in registers across several reflectors (one warp): entries
// i = lane + 32 e of a column segment of length L, zero past L.
template <int E>
__device__ __forceinline__ void load_col(const float* col, int L, float (&x)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        x[e] = i < L ? col[i] : 0.f;
    }
}
template <int E>
__device__ __forceinline__ void store_col(float* col, int L, const float (&x)[E]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i < L) col[i] = x[e];
    }
}

// Householder reflector H = I - tau v v^T of the register column segment
// x[d..L) (d < 32): beta = -sign(x_d) ||x[d..L)||, v = (x - beta e_d) / (x_d - beta)
// so that v[d] = 1 (implicit); entries past d become v, x[d] becomes beta;
// returns tau = (beta - x_d) / beta (0 when x[d+1..L) is zero).  tau and the
// scaling use the fast division: the relative error of a few ulp in tau leaves
// H orthogonal to the FP32 rounding level of the rest of the path.
template <int E>
__device__ __forceinline__ float householder_col(float (&x)[E], int d, int L) {
    const int lane = threadIdx.x & 31;
    float ss0 = 0.f, ss1 = 0.f;                          // two chains: half the dependent latency
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        if (i > d && i < L) {
            if (e & 1) ss1 = fmaf(x[e], x[e], ss1);
            else ss0 = fmaf(x[e], x[e], ss0);
        }
    }
    const float ss = warp_sum(ss0 + ss1);
    const float x0 = __shfl_sync(0xffffffffu, x[0], d);
    float tau = 0.f;
    if (ss > 0.f) {
        const float nrm = sqrtf(fmaf(x0, x0, ss));
        const float beta = -copysignf(nrm, x0);
        // fast divisions (about 2 ulp): H stays orthogonal to the FP32 level
        tau = __fdividef(beta - x0, beta);
        const float scale = __fdividef(1.f, x0 - beta);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = lane + 32 * e;
            if (i > d && i < L) x[e] *= scale;
        }
        if (lane == d) x[0] = beta;
    }
    return tau;
}

// x <- (I - tau v v^T) x for the NC register columns x, with the reflector
// whose diagonal is entry d: v[d] = 1, v[i] = vcol[i] for d < i < L, 0 before d.
template <int E, int NC>
__device__ __forceinline__ void reflect_cols(float (&x)[NC][E], const float* vcol, int d, int L, float tau) {
    const int lane = threadIdx.x & 31;
    float v[E];
    float w[NC], w1[NC];                                  // two chains per column
#pragma unroll
    for (int n = 0; n < NC; ++n) w[n] = w1[n] = 0.f;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int i = lane + 32 * e;
        v[e] = (i > d && i < L) ? vcol[i] : (i == d ? 1.f : 0.f);
#pragma unroll
        for (int n = 0; n < NC; ++n) {
            if (e & 1) w1[n] = fmaf(v[e], x[n][e], w1[n]);
            else w[n] = fmaf(v[e], x[n][e], w[n]);
        }
    }
#pragma unroll
    for (int n = 0; n < NC; ++n) w[n] += w1[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int n = 0; n < NC; ++n) w[n] += __shfl_xor_sync(0xffffffffu, w[n], o);
    }
#pragma unroll
    for (int n = 0; n < NC; ++n) {
        const float wt = w[n] * tau;
#pragma unroll
        for (int e = 0; e < E; ++e) x[n][e] = fmaf(-wt, v[e], x[n][e]);
    }
}

// Named barrier of the kPanel warps that factor a panel (the other warps of
// the CTA do not take part).
__device__ __forceinline__ void panel_bar() {
    asm volatile("bar.sync 1, %0;" ::"r"(kPanel * 32) : "memory");
}

// ---------------------------------------------------------------------------
// One CTA per core: core -> shared memory (column-major, scaled), QR in place,
// R^T -> second region, Jacobi on R^T, norms.  blockIdx.x selects the core
// (core_stride / sigma_stride apart) so one launch serves a batch.

// column stride of the one-CTA kernel's core copy: odd, so the transposing
// copies (lanes along a row of the core) touch 32 different banks
__host__ __device__ __forceinline__ int cta_ldw(int r2) { return r2 | 1; }

template <int NV, int E>
__global__ void __launch_bounds__(kCtaThreads, 1) core_sigma_cta_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, int64_t core_stride,
    double* __restrict__ sigma, int64_t sigma_stride, int* __restrict__ status,
    const int* __restrict__ active, int cert_r1, float cert_ratio, float* __restrict__ vout,
    double* __restrict__ vnorm, int rel_only, int diag_only) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (active && !active[blockIdx.x]) return;
    core += (int64_t)blockIdx.x * core_stride;
    sigma += (int64_t)blockIdx.x * sigma_stride;
    const int sp = 64 * NV;                             // padded column length of R^T (4 x 16 lanes x NV)
    const int ldw = cta_ldw(r2);
    float* W = reinterpret_cast<float*>(smem);          // r2 x s, column-major, column stride ldw
    float* Rt = W + ((size_t)ldw * s + 31) / 32 * 32;   // sp x s, column c = row c of R (128-B aligned)
    __shared__ double s_norm[512];
    __shared__ float s_ptau[2][kPanel], s_red[32];
    __shared__ int s_bad, s_flag;
    __shared__ unsigned int s_meas;
    __shared__ u64 s_dmax;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    // power-of-two scale: largest |entry| -> [0.5, 1)
    if (tid == 0) {
        s_bad = 0;
        s_dmax = 0ull;
    }
    __syncthreads();
    {
        u64 mx = 0ull;
        int bad = 0;
        for (int i = warp; i < r2; i += nwarps) {
            const double* row = core + (int64_t)i * ld;
            for (int j = lane; j < s; j += 32) {
                const u64 ab = abs_bits(row[j]);
                if (ab >= kInfBits) bad = 1;
                else mx = ab > mx ? ab : mx;
            }
        }
        if (bad) s_bad = 1;
        mx = warp_max(mx);
        if (lane == 0) atomicMax(&s_dmax, mx);
    }
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
    for (int i = warp; i < r2; i += nwarps) {
        const double* row = core + (int64_t)i * ld;
        for (int j = lane; j < s; j += 32) W[(size_t)j * ldw + i] = (float)(row[j] * down);
    }
    __syncthreads();

    // Householder QR in panels of kPanel columns with one panel of lookahead.
    // Iteration p: warps 0..kPanel-1 apply the reflectors of panel p to panel
    // p + 1 and factor it (each reflector stays in W below its diagonal, the taus
    // in s_ptau[(p + 1) & 1]); the other warps apply panel p's reflectors to the
    // columns after panel p + 1.  Columns are held in registers (r2 <= 32 E).
    {
        constexpr int NB = kPanel;
        const int np = (s + NB - 1) / NB;
        for (int p = -1; p < np; ++p) {
            if (p >= 0) __syncthreads();
            const int rb = p >= 0 ? p * NB : 0;                // first row held in registers
            const int Lr = r2 - rb;
            const int nxt = p + 1;
            const bool has_next = nxt < np;
            const float* Vp = W + (size_t)(p >= 0 ? p : 0) * NB * ldw + rb;   // reflector c2 at Vp + c2 ldw
            const float* tp = s_ptau[(p >= 0 ? p : 0) & 1];
            if (has_next && warp < NB) {
                const int c = warp;
                const bool has = nxt * NB + c < s;
                float* col = W + (size_t)(nxt * NB + c) * ldw + rb;
                float x[1][E];
                if (has) {
                    load_col<E>(col, Lr, x[0]);
                    if (p >= 0) {
                        for (int c2 = 0; c2 < NB; ++c2) {
                            const float tau = tp[c2];
                            if (tau != 0.f) reflect_cols<E, 1>(x, Vp + (size_t)c2 * ldw, c2, Lr, tau);
                        }
                    }
                }
                const int d0 = nxt * NB - rb;                  // diagonal of the panel's first column
                for (int c2 = 0; c2 < NB; ++c2) {
                    if (c == c2) {
                        float tau = 0.f;
                        if (has) {
                            tau = householder_col<E>(x[0], d0 + c2, Lr);
                            store_col<E>(col, Lr, x[0]);
                        }
                        if (lane == 0) s_ptau[nxt & 1][c2] = tau;
                    }
                    panel_bar();
                    if (c > c2 && has) {
                        const float tau = s_ptau[nxt & 1][c2];
                        if (tau != 0.f) reflect_cols<E, 1>(x, col + (c2 - c) * ldw, d0 + c2, Lr, tau);
                    }
                }
            } else if (p >= 0) {
                // columns after panel p + 1
                const int w0 = has_next ? NB : 0;
                constexpr int NC = E >= 16 ? 1 : 2;
                for (int q = (nxt + 1) * NB + NC * (warp - w0); q < s; q += NC * (nwarps - w0)) {
                    float x[NC][E];
#pragma unroll
                    for (int n = 0; n < NC; ++n) {
                        if (q + n < s) load_col<E>(W + (size_t)(q + n) * ldw + rb, Lr, x[n]);
                        else
#pragma unroll
                            for (int e = 0; e < E; ++e) x[n][e] = 0.f;
                    }
                    for (int c2 = 0; c2 < NB; ++c2) {
                        const float tau = tp[c2];
                        if (tau != 0.f) reflect_cols<E, NC>(x, Vp + (size_t)c2 * ldw, c2, Lr, tau);
                    }
#pragma unroll
                    for (int n = 0; n < NC; ++n)
                        if (q + n < s) store_col<E>(W + (size_t)(q + n) * ldw + rb, Lr, x[n]);
                }
            }
        }
        __syncthreads();
    }
    // The QR-diagonal estimates (the remark after Algorithm 1): |R_kk| sorted, no
    // Jacobi; R_kk = W[k][k] (column-major W holds R in its upper triangle)
    if (diag_only) {
        for (int j = tid; j < s; j += blockDim.x) s_norm[j] = fabs((double)W[(size_t)j * ldw + j]);
        __syncthreads();
        sort_desc(s_norm, s, up, sigma);
        if (tid == 0 && blockIdx.x == 0 && sigma_stride == 0) status[2] = 0;
        if (tid == 0) status[blockIdx.x] = RE_OK;
        return;
    }
    // Certificate of non-convergence (used at intermediate ladder widths only):
    // sigma_r1(core) >= sigma_min(R11) >= 1 / ||R11^{-1}||_F (column interlacing)
    // and sigma_1(core) <= ||R||_F; when the lower bound exceeds cert_ratio times
    // the upper bound, the read-off cannot succeed at this width and the Jacobi
    // sweeps are skipped (status[3] = 1; sigma is not written).
    // (the scratch below needs (1 + min(32, r1)) rounded-up r1 columns of Rt)
    if (cert_r1 > 0 && cert_r1 <= s &&
        (size_t)((cert_r1 + 31) / 32 * 32) * (1 + min(nwarps, cert_r1)) <= (size_t)sp * s) {
        __shared__ float s_fro, s_inv;
        __shared__ int s_zero;
        // Rt is free until the transpose below: 1/R_ii, then one right-hand side per warp
        const int cpad = (cert_r1 + 31) / 32 * 32;
        float* rinv = Rt;
        float* bv = Rt + cpad + (size_t)warp * cpad;
        if (tid == 0) {
            s_fro = 0.f;
            s_inv = 0.f;
            s_zero = 0;
        }
        __syncthreads();
        for (int i = tid; i < cert_r1; i += blockDim.x) {
            const float d = W[(size_t)i * ldw + i];
            rinv[i] = d != 0.f ? 1.f / d : 0.f;
            if (d == 0.f) s_zero = 1;
        }
        float fro = 0.f;
        for (int j = warp; j < s; j += nwarps)
            for (int i = lane; i <= j; i += 32) {
                const float v = W[(size_t)j * ldw + i];
                fro = fmaf(v, v, fro);
            }
        fro = warp_sum(fro);
        if (lane == 0) atomicAdd(&s_fro, fro);
        __syncthreads();
        // columns of R11^{-1} by column-oriented back substitution (R11 x = e_j:
        // x_i = b_i / R_ii, then b[0..i) -= x_i R[0..i, i]; column i of R is
        // contiguous), one warp per column
        float inv = 0.f;
        for (int j = warp; j < cert_r1; j += nwarps) {
            for (int r = lane; r <= j; r += 32) bv[r] = r == j ? 1.f : 0.f;
            __syncwarp();
            float acc = 0.f;
            for (int i = j; i >= 0; --i) {
                const float xi = bv[i] * rinv[i];
                acc = fmaf(xi, xi, acc);
                const float* ci = W + (size_t)i * ldw;
                for (int r = lane; r < i; r += 32) bv[r] = fmaf(-xi, ci[r], bv[r]);
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
    for (int c = warp; c < s; c += nwarps)
        for (int j = lane; j < sp; j += 32)
            Rt[(size_t)c * sp + j] = (j >= c && j < s) ? W[(size_t)j * ldw + c] : 0.f;
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
        const float floor_abs = rel_only ? 0.f : kAbsFloor * s_red[0];
        constexpr int G = 16;
        const int grp = tid / G, ngrp = blockDim.x / G;
        int rotated = 0;
        float meas = 0.f;
        for (int t = 0; t < P - 1; ++t) {
            for (int base = 0; base < P / 2; base += ngrp) {
                if (base + warp * (32 / G) >= P / 2) continue;     // no pair for this warp
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
        if (vout) {
            // right singular vectors of the core: the columns of R^T J, normalised
            const float inv = nv > 0.0 ? (float)(1.0 / nv) : 0.f;
            for (int i = lane; i < s; i += 32) vout[(size_t)j * s + i] = Rt[(size_t)j * sp + i] * inv;
            if (lane == 0) vnorm[j] = nv * up;
        }
    }
    __syncthreads();
    sort_desc(s_norm, s, up, sigma);
    if (tid == 0) status[blockIdx.x] = RE_OK;
}

// ---------------------------------------------------------------------------
// Cluster version: two kernels on the same stream.
//
// core_qr_cluster_kernel (CL CTAs of 512 threads): the columns are dealt out in
// panels of kPanel: panel p (columns p kPanel ..) lives in CTA p % CL as its
// local panel p / CL.  Column stride ldw keeps every column 16-byte aligned.
// The owner of a panel publishes its reflectors once to global memory (each
// panel has its own slot, so no CTA can hold a stale cached copy), and every
// CTA reads them from there (L2, then its L1) after the cluster barrier.  R goes
// to global memory column-major.
//
// core_jacobi_cluster_kernel (CL CTAs of 256 threads, 255 registers per
// thread): blocked one-sided Jacobi on R^T with two column blocks per CTA; in
// the cross rounds each CTA's slot-0 columns stay in registers.

__host__ __device__ __forceinline__ int cluster_ldw(int r2) { return (r2 + 31) / 32 * 32 + 4; }

// Global scratch of the cluster path (floats): R column-major (s x s), the
// reflector slots (np kPanel columns of stride ldw), their taus, and the
// power-of-two scale (one double).
struct ClusterWs {
    float* Rcm;
    float* Vg;
    float* taug;
    double* up;
};
__host__ __device__ __forceinline__ size_t cluster_ws_floats(int r2, int s) {
    const size_t np = (size_t)(s + kPanel - 1) / kPanel;
    return ((size_t)s * s + 3) / 4 * 4 + np * kPanel * (size_t)cluster_ldw(r2) + (np * kPanel + 3) / 4 * 4 + 4;
}
__host__ __device__ __forceinline__ ClusterWs cluster_ws(void* ws, int r2, int s) {
    ClusterWs w;
    const size_t np = (size_t)(s + kPanel - 1) / kPanel;
    w.Rcm = static_cast<float*>(ws);
    w.Vg = w.Rcm + ((size_t)s * s + 3) / 4 * 4;
    w.taug = w.Vg + np * kPanel * (size_t)cluster_ldw(r2);
    w.up = reinterpret_cast<double*>(w.taug + (np * kPanel + 3) / 4 * 4);
    return w;
}

template <int CL, int E>
__global__ void __launch_bounds__(kSvdThreads, 1) core_qr_cluster_kernel(
    const double* __restrict__ core, int r2, int s, int64_t ld, void* ws, double* __restrict__ sigma,
    int* __restrict__ status) {
    constexpr int NB = kPanel;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int np = (s + NB - 1) / NB;                          // panels
    const int nloc = (np + CL - 1) / CL * NB;                  // local columns
    const int ldw = cluster_ldw(r2);
    const ClusterWs g = cluster_ws(ws, r2, s);
    float* W = reinterpret_cast<float*>(smem);                // nloc columns, stride ldw
    __shared__ float s_ptau[NB];
    __shared__ int s_bad;
    __shared__ u64 s_dmax;
    const int k = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    // global column of local column jl
    auto gcol = [&](int jl) { return ((jl / NB) * CL + k) * NB + (jl % NB); };

    // ---- own columns: finiteness and the power-of-two scale agreed across the cluster
    if (tid == 0) {
        s_bad = 0;
        s_dmax = 0ull;
    }
    __syncthreads();
    {
        u64 mx = 0ull;
        int bad = 0;
        for (int i = warp; i < r2; i += nwarps) {
            const double* row = core + (int64_t)i * ld;
            for (int jl = lane; jl < nloc; jl += 32) {
                const int j = gcol(jl);
                if (j < s) {
                    const u64 ab = abs_bits(row[j]);
                    if (ab >= kInfBits) bad = 1;
                    else mx = ab > mx ? ab : mx;
                }
            }
        }
        if (bad) s_bad = 1;
        mx = warp_max(mx);
        if (lane == 0) atomicMax(&s_dmax, mx);
    }
    cluster.sync();
    int any_bad = 0;
    u64 gbits = 0ull;
    for (int r = 0; r < CL; ++r) {
        any_bad |= *cluster.map_shared_rank(&s_bad, r);
        const u64 m = *cluster.map_shared_rank(&s_dmax, r);
        gbits = m > gbits ? m : gbits;
    }
    if (any_bad) {
        if (k == 0) {
            for (int j = tid; j < s; j += blockDim.x) sigma[j] = nan("");
            if (tid == 0) *status = RE_ERR_NONFINITE;
        }
        cluster.sync();
        return;
    }
    const double gmax = __longlong_as_double((long long)gbits);
    int e2 = 0;
    if (gmax > 0.0) frexp(gmax, &e2);
    const double down = ldexp(1.0, -e2);
    if (k == 0 && tid == 0) {
        *g.up = ldexp(1.0, e2);
        *status = RE_OK;
    }
    for (int i = warp; i < ldw; i += nwarps) {
        const double* row = core + (int64_t)i * ld;
        for (int jl = lane; jl < nloc; jl += 32) {
            const int j = gcol(jl);
            W[(size_t)jl * ldw + i] = (i < r2 && j < s) ? (float)(row[j] * down) : 0.f;
        }
    }
    cluster.sync();   // all CTAs have read every s_bad / s_dmax

    // ---- panel Householder QR with one panel of lookahead.  Iteration p: the
    // reflectors V_p of panel p are in global slot p (published before the
    // barrier); the owner of panel p + 1 applies V_p to that panel, factors it and
    // publishes its reflectors in slot p + 1, while every other warp applies V_p to
    // the trailing columns of its CTA.
    for (int p = -1; p < np; ++p) {
        if (p >= 0) cluster.sync();
        const int rb = p >= 0 ? p * NB : 0;                    // first row held in registers
        const int Lr = r2 - rb;
        const int nxt = p + 1;
        const bool own_next = nxt < np && k == nxt % CL;
        const float* Vp = g.Vg + (size_t)(p >= 0 ? p : 0) * NB * ldw + rb;
        const float* tp = g.taug + (size_t)(p >= 0 ? p : 0) * NB;
        if (p >= 0) {
            // request every line of V_p and its taus at once: the reflector loads
            // below then hit L1 instead of paying one L2 round trip each
            const int lpc = (Lr + 31) / 32 + 1;                // 128-byte steps per column
            for (int i = tid; i < NB * lpc + 1; i += blockDim.x) {
                const float* a = i < NB * lpc ? Vp + (size_t)(i / lpc) * ldw + 32 * (i % lpc) : tp;
                asm volatile("prefetch.L1 [%0];" ::"l"(a));
            }
        }
        if (own_next && warp < NB) {
            const int c = warp;
            const int lc = (nxt / CL) * NB + c;
            float* col = W + (size_t)lc * ldw + rb;
            float x[1][E];
            load_col<E>(col, Lr, x[0]);
            if (p >= 0) {
                for (int c2 = 0; c2 < NB; ++c2) {
                    const float tau = tp[c2];
                    if (tau != 0.f) reflect_cols<E, 1>(x, Vp + (size_t)c2 * ldw, c2, Lr, tau);
                }
            }
            const int d0 = nxt * NB - rb;                      // diagonal of the panel's first column
            for (int c2 = 0; c2 < NB; ++c2) {
                if (c == c2) {
                    const float tau = householder_col<E>(x[0], d0 + c2, Lr);
                    store_col<E>(col, Lr, x[0]);
                    if (lane == 0) s_ptau[c2] = tau;
                }
                panel_bar();
                if (c > c2) {
                    const float tau = s_ptau[c2];
                    if (tau != 0.f) reflect_cols<E, 1>(x, col + (c2 - c) * ldw, d0 + c2, Lr, tau);
                }
            }
            // publish this column's rows [nxt NB, r2) and its tau in slot nxt
            const float4* src = reinterpret_cast<const float4*>(W + (size_t)lc * ldw);
            float4* dst = reinterpret_cast<float4*>(g.Vg + ((size_t)nxt * NB + c) * ldw);
            for (int q = nxt * NB / 4 + lane; q < (r2 + 3) / 4; q += 32) dst[q] = src[q];
            if (lane == 0) g.taug[(size_t)nxt * NB + c] = s_ptau[c];
            __threadfence();
        } else if (p >= 0) {
            // trailing columns of this CTA: local panels whose global panel is > p
            int lp0 = p >= k ? (p - k) / CL + 1 : 0;
            if (own_next) ++lp0;                               // panel p + 1 is with warps < NB
            const int w0 = own_next ? NB : 0;
            constexpr int NC = E >= 32 ? 1 : 2;
            for (int q = lp0 * NB + NC * (warp - w0); q < nloc; q += NC * (nwarps - w0)) {
                float x[NC][E];
                bool ok[NC];
#pragma unroll
                for (int n = 0; n < NC; ++n) {
                    ok[n] = q + n < nloc && gcol(q + n) < s;   // padding columns stay zero
                    if (ok[n]) load_col<E>(W + (size_t)(q + n) * ldw + rb, Lr, x[n]);
                    else
#pragma unroll
                        for (int e = 0; e < E; ++e) x[n][e] = 0.f;
                }
                for (int c2 = 0; c2 < NB; ++c2) {
                    const float tau = tp[c2];
                    if (tau != 0.f) reflect_cols<E, NC>(x, Vp + (size_t)c2 * ldw, c2, Lr, tau);
                }
#pragma unroll
                for (int n = 0; n < NC; ++n)
                    if (ok[n]) store_col<E>(W + (size_t)(q + n) * ldw + rb, Lr, x[n]);
            }
        }
    }
    __syncthreads();
    // ---- R (upper triangle of the first s rows) to global, column-major
    for (int jl = warp; jl < nloc; jl += nwarps) {
        const int j = gcol(jl);
        if (j >= s) continue;
        for (int i = lane; i <= j; i += 32) g.Rcm[(size_t)j * s + i] = W[(size_t)jl * ldw + i];
    }
}

// Cross pairs of one tournament round: in inner round u, column j of slot 0 (c0)
// meets column (j+u) mod b of slot 1 (c1).  Column j (lane group j; b <= groups
// per CTA) stays in registers for the b inner rounds, the slot-1 columns pass
// through shared memory; at the end column j is written to x_dst + j sp.
template <int G, int NVG>
__device__ __forceinline__ void cross_rounds(const float* c0, float* c1, float* x_dst, int b, int sp, float tol2,
                                             float floor_abs, float& meas, int& rotated) {
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid / G, gl = tid & (G - 1);
    const bool wact = warp * (32 / G) < b;                  // warp holds a slot-0 column
    const int j = grp;
    const bool act = j < b;
    ulonglong2 x[NVG];
    if (act) {
#pragma unroll
        for (int v = 0; v < NVG; ++v) x[v] = *reinterpret_cast<const ulonglong2*>(c0 + (size_t)j * sp + 4 * (gl + G * v));
    }
    for (int u = 0; u < b; ++u) {
        if (wact) {
            int jj = act ? j + u : 0;
            if (jj >= b) jj -= b;
            jacobi_pair_x<G, NVG>(act, x, c1 + (size_t)jj * sp, tol2, floor_abs, meas, rotated);
        }
        __syncthreads();
    }
    if (act) {   // slot-0 column j to its next place (possibly another CTA's shared memory)
#pragma unroll
        for (int v = 0; v < NVG; ++v) *reinterpret_cast<ulonglong2*>(x_dst + (size_t)j * sp + 4 * (gl + G * v)) = x[v];
    }
}

// lanes per column pair of the cluster Jacobi: 8 (fewer shuffle levels) while
// the register-held columns fit, 16 for the longest columns
__host__ __device__ constexpr int jac_g(int nq) { return nq >= 4 ? 16 : 8; }

template <int CL, int NQ>
__global__ void __launch_bounds__(kJacThreads, 1) core_jacobi_cluster_kernel(
    const void* ws, int r2, int s, int b, double* __restrict__ sigma, int* __restrict__ status,
    float* __restrict__ vout, double* __restrict__ vnorm, int rel_only) {
    constexpr int P2 = 2 * CL;
    constexpr int G = jac_g(NQ);                               // lanes per column pair
    constexpr int NVG = 32 * NQ / G;                           // float4 per lane per column
    constexpr int GPW = 32 / G;                                // pair groups per warp
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int sp = 128 * NQ;                                   // padded column length of R^T
    const size_t set_floats = 2 * (size_t)b * sp;              // two blocks of b columns
    float* const set0 = reinterpret_cast<float*>(smem);
    auto sets = [&](int i) { return i ? set0 + set_floats : set0; };   // Jacobi ping-pong
    __shared__ int s_count;
    __shared__ unsigned int s_meas;
    __shared__ float s_fmax;
    __shared__ double s_norm[512];
    __shared__ float s_red[32];
    const int k = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const ClusterWs g = cluster_ws(const_cast<void*>(ws), r2, s);
    if (*status == RE_ERR_NONFINITE) return;                   // the QR kernel found Inf/NaN (uniform)

    if (tid == 0) {
        s_count = 0;
        s_meas = 0u;
    }
    // ---- the two R^T column blocks of this CTA (positions k and P2-1-k): column
    // c = row c of R, read from R column-major (16 consecutive rows per column)
    for (int sl = 0; sl < 2; ++sl) {
        const int blk = sl == 0 ? k : P2 - 1 - k;
        float* dst = sets(0) + (size_t)sl * b * sp;
        for (int idx = tid; idx < b * sp; idx += blockDim.x) {
            const int jj = idx % b, col = idx / b;             // jj fastest: consecutive rows of R
            const int c = blk * b + jj;
            float val = 0.f;
            if (c < s && col >= c && col < s) val = g.Rcm[(size_t)col * s + c];
            dst[(size_t)jj * sp + col] = val;
        }
    }
    __syncthreads();
    cluster.sync();

    // ---- blocked Jacobi on R^T (length-sp columns, zero padded)
    const float tol = 4.f * kU * sqrtf((float)s);
    const int grp = tid / G, ngrp = blockDim.x / G;
    int cur = 0;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        float amax = 0.f;
        for (int q = warp; q < 2 * b; q += nwarps) {
            const float* a = sets(cur) + (size_t)q * sp;
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
        const float floor_abs = rel_only ? 0.f : kAbsFloor * gm;
        int rotated = 0;
        float meas = 0.f;
        for (int t = 0; t < P2 - 1; ++t) {
            float* c0 = sets(cur);
            float* c1 = c0 + (size_t)b * sp;
            if (t == 0) {
                // pairs inside each block (circle ordering on b columns)
                const int P = b + (b & 1);
                for (int u = 0; u < P - 1; ++u) {
                    for (int base = 0; base < P; base += ngrp) {
                        if (base + warp * GPW >= P) continue;    // no pair for this warp
                        const int q = base + grp;
                        bool act = q < P;
                        float* pa = c0;
                        float* pb = c0;
                        if (act) {
                            const int sl = q / (P / 2), kq = q % (P / 2);
                            const int e1 = circle_player(kq, u, P), e2 = circle_player(P - 1 - kq, u, P);
                            const int pp = min(e1, e2), qq = max(e1, e2);
                            act = qq < b;
                            float* bs = sl == 0 ? c0 : c1;
                            pa = bs + (size_t)pp * sp;
                            pb = bs + (size_t)qq * sp;
                        }
                        jacobi_pair<G, NVG>(act, pa, pb, tol * tol, floor_abs, meas, rotated);
                    }
                    __syncthreads();
                }
            }
            // tournament positions 1..P2-1 move up by one, position 0 stays (slot 0 of
            // CTA k is position k, slot 1 is position P2-1-k): each CTA pushes its two
            // blocks into the other set of the CTAs holding their next positions; that
            // set was last used in the previous round, before the barrier below
            const int nxt = cur ^ 1;
            const int d0 = k == 0 ? 0 : (k < CL - 1 ? k + 1 : CL - 1);
            const int sl0 = k == CL - 1 ? 1 : 0;
            const int d1 = k == 0 ? 1 : k - 1;
            const int sl1 = k == 0 ? 0 : 1;
            float* x_dst = cluster.map_shared_rank(sets(nxt) + (size_t)sl0 * b * sp, d0);
            cross_rounds<G, NVG>(c0, c1, x_dst, b, sp, tol * tol, floor_abs, meas, rotated);
            {
                const float4* from = reinterpret_cast<const float4*>(c1);
                float4* to = reinterpret_cast<float4*>(cluster.map_shared_rank(sets(nxt) + (size_t)sl1 * b * sp, d1));
                const int n4 = b * sp / 4;
                for (int i = tid; i < n4; i += kJacThreads) to[i] = from[i];
            }
            cluster.sync();
            cur = nxt;
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
    // ---- norms gathered in CTA 0
    for (int q = warp; q < 2 * b; q += nwarps) {
        const int sl = q / b, j = q % b;
        const int c = (sl == 0 ? k : P2 - 1 - k) * b + j;   // a whole sweep returns every block home
        const double nv = col_norm(sets(cur) + (size_t)q * sp, sp);
        if (lane == 0 && c < s) *cluster.map_shared_rank(&s_norm[c], 0) = nv;
        if (vout && c < s) {
            // right singular vectors of the core: the columns of R^T J, normalised
            const float inv = nv > 0.0 ? (float)(1.0 / nv) : 0.f;
            const float* col = sets(cur) + (size_t)q * sp;
            for (int i = lane; i < s; i += 32) vout[(size_t)c * s + i] = col[i] * inv;
            if (lane == 0) vnorm[c] = nv * *g.up;
        }
    }
    cluster.sync();
    if (k == 0) {
        sort_desc(s_norm, s, *g.up, sigma);
        if (tid == 0) *status = RE_OK;
    }
}

size_t qr_cluster_smem(int CL, int r2, int s) {
    const int np = (s + kPanel - 1) / kPanel;
    const size_t nloc = (size_t)(np + CL - 1) / CL * kPanel;
    return sizeof(float) * nloc * (size_t)cluster_ldw(r2);
}
size_t jac_cluster_smem(int CL, int s, int* b_out) {
    const int b = (s + 2 * CL - 1) / (2 * CL);
    const size_t sp = (size_t)(s + 127) / 128 * 128;
    *b_out = b;
    return sizeof(float) * 4 * (size_t)b * sp;
}

template <int CL>
cudaError_t set_cluster_attrs(const void* kern, size_t smem) {
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e == cudaSuccess && CL > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int CL, class... Args>
cudaError_t launch_cluster(void (*kern)(Args...), int threads, size_t smem, cudaStream_t st, Args... args) {
    cudaError_t e = set_cluster_attrs<CL>(reinterpret_cast<const void*>(kern), smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int CL>
cudaError_t launch_qr_cluster(const double* core, int r2, int s, int64_t ld, void* ws, double* sigma, int* status,
                              cudaStream_t st) {
    const size_t smem = qr_cluster_smem(CL, r2, s);
    const int e = (r2 + 31) / 32;                             // column length r2 <= 32 E
    if (e <= 8)
        return launch_cluster<CL>(core_qr_cluster_kernel<CL, 8>, kSvdThreads, smem, st, core, r2, s, ld, ws, sigma,
                                  status);
    if (e <= 16)
        return launch_cluster<CL>(core_qr_cluster_kernel<CL, 16>, kSvdThreads, smem, st, core, r2, s, ld, ws, sigma,
                                  status);
    if (e <= 32)
        return launch_cluster<CL>(core_qr_cluster_kernel<CL, 32>, kSvdThreads, smem, st, core, r2, s, ld, ws, sigma,
                                  status);
    return cudaErrorInvalidValue;
}

template <int CL>
cudaError_t launch_jacobi_cluster(void* ws, int r2, int s, double* sigma, int* status, cudaStream_t st, float* vout,
                                  double* vnorm, int rel_only) {
    int b = 0;
    const size_t smem = jac_cluster_smem(CL, s, &b);
    const void* cws = ws;
    const int nq = (s + 127) / 128;
    if (nq < 1 || nq > 4 || b > kJacThreads / jac_g(nq)) return cudaErrorInvalidValue;   // one lane group per slot-0 column
    switch (nq) {
        case 1: return launch_cluster<CL>(core_jacobi_cluster_kernel<CL, 1>, kJacThreads, smem, st, cws, r2, s, b, sigma, status, vout, vnorm, rel_only);
        case 2: return launch_cluster<CL>(core_jacobi_cluster_kernel<CL, 2>, kJacThreads, smem, st, cws, r2, s, b, sigma, status, vout, vnorm, rel_only);
        case 3: return launch_cluster<CL>(core_jacobi_cluster_kernel<CL, 3>, kJacThreads, smem, st, cws, r2, s, b, sigma, status, vout, vnorm, rel_only);
        case 4: return launch_cluster<CL>(core_jacobi_cluster_kernel<CL, 4>, kJacThreads, smem, st, cws, r2, s, b, sigma, status, vout, vnorm, rel_only);
        default: return cudaErrorInvalidValue;
    }
}

// The QR-diagonal estimates after the cluster QR: |R_kk| of R (column-major in the
// workspace), sorted descending and scaled back (one CTA).
__global__ void qrdiag_cluster_kernel(const void* ws, int r2, int s, double* __restrict__ sigma,
                                      int* __restrict__ status) {
    __shared__ double s_norm[512];
    if (*status == RE_ERR_NONFINITE) return;
    const ClusterWs g = cluster_ws(const_cast<void*>(ws), r2, s);
    for (int j = threadIdx.x; j < s; j += blockDim.x) s_norm[j] = fabs((double)g.Rcm[(size_t)j * s + j]);
    __syncthreads();
    sort_desc(s_norm, s, *g.up, sigma);
    if (threadIdx.x == 0) {
        status[2] = 0;
        *status = RE_OK;
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
    return sizeof(float) * (((size_t)cta_ldw(r2) * s + 31) / 32 * 32 + sp * s);
}

}  // namespace

size_t svd_workspace_bytes(int r2, int s) { return sizeof(float) * cluster_ws_floats(r2, s) + 256; }

namespace {

using CtaKernel = void (*)(const double*, int, int, int64_t, int64_t, double*, int64_t, int*, const int*, int,
                           float, float*, double*, int, int);

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
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern));
    if (e != cudaSuccess) return e;
    // many small cores: 512 threads (8 panel + 8 trailing warps, 32 pair groups) fit
    // two CTAs in an SM's registers where 1024 fit one; every loop of the kernel
    // takes its warp and group counts from the launch
    const int threads = (count > 1 && s <= 64) ? 512 : kCtaThreads;
    kern<<<count, threads, sm, st>>>(core, r2, s, ld, core_stride, sigma, sigma_stride, status, active,
                                     cert_r1, cert_ratio, nullptr, nullptr, 0, 0);
    return cudaGetLastError();
}

namespace {

// The single-core path with the optional outputs of the precision mode: the
// normalised Jacobi columns (vout, s x s column-major, unsorted) with their
// norms, and rel_only (no absolute rotation floor).
cudaError_t core_sigma_one(const double* core, int r2, int s, int64_t ld, void* ws, double* sigma, int* status,
                           cudaStream_t st, int cert_r1, float cert_ratio, float* vout, double* vnorm,
                           int rel_only, int diag_only = 0) {
    if (s <= 0) return cudaSuccess;
    if (s > 512) return cudaErrorInvalidValue;
    if (cta_smem(r2, s) <= kSmemLimit) {
        const size_t sm = cta_smem(r2, s);
        auto kern = cta_kernel_for((s + 63) / 64, (r2 + 31) / 32);
        if (!kern) return cudaErrorInvalidValue;
        cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(kern));
        if (e != cudaSuccess) return e;
        kern<<<1, kCtaThreads, sm, st>>>(core, r2, s, ld, 0, sigma, 0, status, nullptr, cert_r1, cert_ratio, vout,
                                         vnorm, rel_only, diag_only);
        return cudaGetLastError();
    }
    // larger cores: QR on a cluster, then Jacobi on a cluster; ws holds
    // svd_workspace_bytes(r2, s) (16-byte aligned)
    if (!ws) return cudaErrorInvalidValue;
    cudaError_t e;
    if (qr_cluster_smem(8, r2, s) <= kSmemLimit) e = launch_qr_cluster<8>(core, r2, s, ld, ws, sigma, status, st);
    else if (qr_cluster_smem(16, r2, s) <= kSmemLimit) e = launch_qr_cluster<16>(core, r2, s, ld, ws, sigma, status, st);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    if (diag_only) {
        qrdiag_cluster_kernel<<<1, 512, 0, st>>>(ws, r2, s, sigma, status);
        return cudaGetLastError();
    }
    int b = 0;
    if (jac_cluster_smem(8, s, &b) <= kSmemLimit)
        return launch_jacobi_cluster<8>(ws, r2, s, sigma, status, st, vout, vnorm, rel_only);
    if (jac_cluster_smem(16, s, &b) <= kSmemLimit)
        return launch_jacobi_cluster<16>(ws, r2, s, sigma, status, st, vout, vnorm, rel_only);
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_core_sigma(const double* core, int r2, int s, int64_t ld, void* ws, double* sigma,
                              int* status, cudaStream_t st, int cert_r1, float cert_ratio) {
    return core_sigma_one(core, r2, s, ld, ws, sigma, status, st, cert_r1, cert_ratio, nullptr, nullptr, 0);
}

cudaError_t launch_core_qrdiag(const double* core, int r2, int s, int64_t ld, void* ws, double* sigma, int* status,
                               cudaStream_t st) {
    return core_sigma_one(core, r2, s, ld, ws, sigma, status, st, 0, 0.f, nullptr, nullptr, 0, 1);
}

namespace {

// perm[rank] = j, ranks by descending vnorm (ties: smaller j first); one CTA.
__global__ void norm_order_kernel(const double* __restrict__ vnorm, int s, int* __restrict__ perm) {
    for (int j = threadIdx.x; j < s; j += blockDim.x) {
        const long long vb = __double_as_longlong(vnorm[j]);
        int rank = 0;
        for (int i = 0; i < s; ++i) {
            const long long w = __double_as_longlong(vnorm[i]);
            rank += (w > vb) || (w == vb && i < j);
        }
        perm[rank] = j;
    }
}

// W = C V(:, perm) in FP64 (C r2 x s row-major with ld; V s x s column-major FP32,
// exact in FP64): 32 x 32 output tiles, K tiles of 32, four outputs per thread.
__global__ void __launch_bounds__(256) precond_gemm_kernel(const double* __restrict__ C, int64_t ld, int r2, int s,
                                                           const float* __restrict__ V, const int* __restrict__ perm,
                                                           double* __restrict__ W, int64_t ldw) {
    __shared__ double cs[32][33], vs[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // ty 0..7
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int jcol = j0 + tx < s ? perm[j0 + tx] : 0;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = 0; k0 < s; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int i = i0 + r, k = k0 + tx;
            cs[r][tx] = (i < r2 && k < s) ? C[(int64_t)i * ld + k] : 0.0;
            // vs[k][j]: column perm[j0 + r] of V, row k0 + tx
            const int jj = j0 + r;
            vs[tx][r] = (jj < s && k < s) ? (double)V[(size_t)perm[jj] * s + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            const double v = vs[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(cs[ty + 8 * q][k], v, acc[q]);
        }
        __syncthreads();
    }
    (void)jcol;
    if (j0 + tx < s)
        for (int q = 0; q < 4; ++q) {
            const int i = i0 + ty + 8 * q;
            if (i < r2) W[(int64_t)i * ldw + j0 + tx] = acc[q];
        }
}

}  // namespace

size_t svd_precise_bytes(int r2, int s) {
    const size_t v = ((size_t)s * s * sizeof(float) + 255) / 256 * 256;
    const size_t n = ((size_t)s * sizeof(double) + 255) / 256 * 256;
    const size_t pm = ((size_t)s * sizeof(int) + 255) / 256 * 256;
    const size_t w = ((size_t)r2 * s * sizeof(double) + 255) / 256 * 256;
    return v + n + pm + w;
}

cudaError_t launch_core_sigma_precise(const double* core, int r2, int s, int64_t ld, void* ws, void* pws,
                                      double* sigma, int* status, cudaStream_t st) {
    if (s <= 0) return cudaSuccess;
    if (s > 512 || !pws) return cudaErrorInvalidValue;
    char* b = static_cast<char*>(pws);
    float* V = reinterpret_cast<float*>(b);
    b += ((size_t)s * s * sizeof(float) + 255) / 256 * 256;
    double* vnorm = reinterpret_cast<double*>(b);
    b += ((size_t)s * sizeof(double) + 255) / 256 * 256;
    int* perm = reinterpret_cast<int*>(b);
    b += ((size_t)s * sizeof(int) + 255) / 256 * 256;
    double* W = reinterpret_cast<double*>(b);
    // stage 1: FP32 QR + Jacobi of the core, keeping its right singular vectors V1;
    // every pair is orthogonalised (no absolute floor), so V1 is orthogonal to
    // working precision in its small-value columns too
    cudaError_t e = core_sigma_one(core, r2, s, ld, ws, sigma, status, st, 0, 0.f, V, vnorm, 1);
    if (e != cudaSuccess) return e;
    norm_order_kernel<<<1, 512, 0, st>>>(vnorm, s, perm);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // stage 2: W = core V1 in FP64; its columns are graded (nearly sigma_k u_k)
    dim3 grid((unsigned)((s + 31) / 32), (unsigned)((r2 + 31) / 32));
    precond_gemm_kernel<<<grid, 256, 0, st>>>(core, ld, r2, s, V, perm, W, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // stage 3: FP32 QR + Jacobi of W with the relative rotation test only
    return core_sigma_one(W, r2, s, s, ws, sigma, status, st, 0, 0.f, nullptr, nullptr, 1);
}

cudaError_t launch_readoff(const double* sigma, int r1, double scale, double eps, double norm_a,
                           const int* status_in, DevReadoff* out, double* sigma_scaled,
                           cudaStream_t st) {
    readoff_kernel<<<1, 32, 0, st>>>(sigma, r1, scale, eps, norm_a, status_in, out, sigma_scaled);
    return cudaGetLastError();
}

}  // namespace re
