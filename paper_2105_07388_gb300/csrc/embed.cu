// Random embeddings X and Y drawn from the counter-based generator (common.cuh):
// Gaussian G (Sec. 1 notation; Sec. 3.4) and the SRTT ingredients D and S of
// Eq. (Theta) (Sec. 4).  The Gaussian right embedding is written once per sketch
// step into a small buffer (n x s, L2-resident) that the right-sketch kernels
// stream; the left embedding Y is generated inside the left-sketch kernel and
// is only written out here for re_embedding_y.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

// One thread per (row k, column group g): X[k][4g+t] = normal t of Philox(k, g, GX).
__global__ void gauss_x_kernel(uint64_t seed, int64_t n, int g0, int ng, int col0, int s, float* X,
                               int64_t ldx) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * ng) return;
    const int64_t k = idx / ng;
    const int g = g0 + (int)(idx % ng);
    float z[4];
    normals4((uint32_t)k, (uint32_t)g, kStreamGX, seed, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = 4 * g + t - col0;
        if (j >= 0 && j < s) X[k * ldx + j] = z[t];
    }
}

// Transposed BF16 copy for the tensor-core path: Xt[j][k] (k contiguous); rows
// k in [n, n_alloc) are zero so full K tiles can be read past the edge.
__global__ void gauss_xt_bf16_kernel(uint64_t seed, int64_t n, int64_t n_alloc, int g0, int ng,
                                     int col0, int s, uint16_t* Xt, int64_t ldt) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_alloc * ng) return;
    const int64_t k = idx % n_alloc;
    const int g = g0 + (int)(idx / n_alloc);
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (k < n) normals4((uint32_t)k, (uint32_t)g, kStreamGX, seed, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int j = 4 * g + t - col0;
        if (j >= 0 && j < s) Xt[(int64_t)j * ldt + k] = (uint16_t)(__float_as_uint(z[t]) >> 16);
    }
}

// Xt[j][k] (BF16 bits) = d_k H[k][cols[j]] for k < n, 0 for n <= k < n_alloc: the
// SRTT right embedding's sampled columns, +-1 and exact in BF16.
__global__ void srht_xt_bf16_kernel(int64_t n, int64_t n_alloc, const int* __restrict__ cols,
                                    const uint32_t* __restrict__ dbits, int s, uint16_t* __restrict__ Xt,
                                    int64_t ldt) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_alloc * s) return;
    const int64_t k = idx % n_alloc;
    const int j = (int)(idx / n_alloc);
    uint16_t v = 0;
    if (k < n) {
        const uint32_t neg = ((dbits[k >> 5] >> (k & 31)) ^ (uint32_t)__popcll((unsigned long long)k &
                                                                              (unsigned long long)cols[j])) & 1u;
        v = neg ? (uint16_t)0xBF80u : (uint16_t)0x3F80u;      // -1 / +1
    }
    Xt[(int64_t)j * ldt + k] = v;
}

__global__ void gauss_y_kernel(uint64_t seed, int64_t m, int g0, int ng, int row0, int r2, float* Y,
                               int64_t ldy) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * ng) return;
    const int64_t i = idx % m;
    const int g = g0 + (int)(idx / m);
    float z[4];
    normals4((uint32_t)i, (uint32_t)g, kStreamGY, seed, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int q = 4 * g + t - row0;
        if (q >= 0 && q < r2) Y[(int64_t)q * ldy + i] = z[t];
    }
}

// words[w] bit b  <=>  d_{32w+b} = -1; Philox(j/128, 0, stream, 0) supplies j mod 128.
__global__ void sign_bits_kernel(uint64_t seed, uint32_t stream, int64_t nwords, int64_t count,
                                 uint32_t* words) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nwords) return;
    const U4 r = philox((uint32_t)(w >> 2), 0u, stream, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const int sel = (int)(w & 3);
    uint32_t v = sel == 0 ? r.x : sel == 1 ? r.y : sel == 2 ? r.z : r.w;
    const int64_t first = w * 32;
    if (first + 32 > count) {
        const int keep = (int)(count - first);
        v = keep <= 0 ? 0u : (keep >= 32 ? v : (v & ((1u << keep) - 1u)));
    }
    words[w] = v;
}

__global__ void perm_kernel(uint64_t seed, uint32_t stream, int bits, int k0, int cnt, int* out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    out[k] = (int)feistel((uint32_t)(k0 + k), bits, stream, seed);
}

__global__ void srtt_x_dense_kernel(int64_t n, int s, const uint32_t* dbits, const int* cols,
                                    float* X, int64_t ldx) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * s) return;
    const int64_t k = idx / s;
    const int j = (int)(idx % s);
    const uint32_t par = (__popcll((unsigned long long)(k & (int64_t)cols[j])) & 1) ^
                         ((dbits[k >> 5] >> (k & 31)) & 1u);
    X[k * ldx + j] = par ? -1.0f : 1.0f;
}

// HRTT hashing table (Sec. 3.4): entry q is c = pi_X(q) with bit 15 set when the
// CountSketch sign sigma_c (stream SX, drawn as the SRTT signs) is -1.  Bucket k
// of width s is {entry q : q = k mod s}, so one table serves every width.
__global__ void hrtt_table_kernel(uint64_t seed, int bits, int np, uint16_t* tbl) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    const uint32_t c = feistel((uint32_t)q, bits, kStreamPX, seed);
    const U4 r = philox(c >> 7, 0u, kStreamSX, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    const int sel = (int)((c & 127u) >> 5);
    const uint32_t w = sel == 0 ? r.x : sel == 1 ? r.y : sel == 2 ? r.z : r.w;
    tbl[q] = (uint16_t)(c | (((w >> (c & 31u)) & 1u) << 15));
}

// Dense HRTT X (n x s, entries are sums of +-1, exact in FP32):
// X[k, j] = d_k sum over bucket j of sigma_c H[k, c].
__global__ void hrtt_x_dense_kernel(int64_t n, int s, int np, const uint32_t* dbits, const uint16_t* tbl,
                                    float* X, int64_t ldx) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * s) return;
    const int64_t k = idx / s;
    const int j = (int)(idx % s);
    int acc = 0;
    for (int q = j; q < np; q += s) {
        const uint32_t e = tbl[q];
        const uint32_t par = (__popcll((unsigned long long)(k & (int64_t)(e & 0x7fffu))) & 1) ^ (e >> 15);
        acc += par ? -1 : 1;
    }
    X[k * ldx + j] = ((dbits[k >> 5] >> (k & 31)) & 1u) ? (float)-acc : (float)acc;
}

__global__ void srtt_y_dense_kernel(int64_t m, int r2, const uint32_t* dbits, const int* rows,
                                    float* Y, int64_t ldy) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * r2) return;
    const int q = (int)(idx / m);
    const int64_t i = idx % m;
    const uint32_t par = (__popcll((unsigned long long)(i & (int64_t)rows[q])) & 1) ^
                         ((dbits[i >> 5] >> (i & 31)) & 1u);
    Y[(int64_t)q * ldy + i] = par ? -1.0f : 1.0f;
}

inline unsigned blocks_for(int64_t total, int threads) {
    return (unsigned)((total + threads - 1) / threads);
}

}  // namespace

cudaError_t launch_gauss_x(uint64_t seed, int64_t n, int col0, int s, float* X, int64_t ldx,
                           cudaStream_t st) {
    if (n <= 0 || s <= 0) return cudaSuccess;
    const int g0 = col0 / 4, g1 = (col0 + s + 3) / 4, ng = g1 - g0;
    gauss_x_kernel<<<blocks_for(n * ng, 256), 256, 0, st>>>(seed, n, g0, ng, col0, s, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_gauss_xt_bf16(uint64_t seed, int64_t n, int64_t n_alloc, int col0, int s,
                                 uint16_t* Xt, int64_t ldt, cudaStream_t st) {
    if (n_alloc <= 0 || s <= 0) return cudaSuccess;
    const int g0 = col0 / 4, g1 = (col0 + s + 3) / 4, ng = g1 - g0;
    gauss_xt_bf16_kernel<<<blocks_for(n_alloc * ng, 256), 256, 0, st>>>(seed, n, n_alloc, g0, ng,
                                                                         col0, s, Xt, ldt);
    return cudaGetLastError();
}

cudaError_t launch_srht_xt_bf16(int64_t n, int64_t n_alloc, const int* cols, const uint32_t* dbits, int s,
                                uint16_t* Xt, int64_t ldt, cudaStream_t st) {
    if (n_alloc <= 0 || s <= 0) return cudaSuccess;
    srht_xt_bf16_kernel<<<blocks_for(n_alloc * s, 256), 256, 0, st>>>(n, n_alloc, cols, dbits, s, Xt, ldt);
    return cudaGetLastError();
}

cudaError_t launch_gauss_y(uint64_t seed, int64_t m, int row0, int r2, float* Y, int64_t ldy,
                           cudaStream_t st) {
    if (m <= 0 || r2 <= 0) return cudaSuccess;
    const int g0 = row0 / 4, g1 = (row0 + r2 + 3) / 4, ng = g1 - g0;
    gauss_y_kernel<<<blocks_for(m * ng, 256), 256, 0, st>>>(seed, m, g0, ng, row0, r2, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_sign_bits(uint64_t seed, uint32_t stream, int64_t count, uint32_t* words,
                             cudaStream_t st) {
    const int64_t nwords = (count + 31) / 32;
    if (nwords <= 0) return cudaSuccess;
    sign_bits_kernel<<<blocks_for(nwords, 256), 256, 0, st>>>(seed, stream, nwords, count, words);
    return cudaGetLastError();
}

cudaError_t launch_perm(uint64_t seed, uint32_t stream, int bits, int k0, int cnt, int* out,
                        cudaStream_t st) {
    if (cnt <= 0) return cudaSuccess;
    perm_kernel<<<blocks_for(cnt, 256), 256, 0, st>>>(seed, stream, bits, k0, cnt, out);
    return cudaGetLastError();
}

cudaError_t launch_srtt_x_dense(int64_t n, int s, const uint32_t* dbits, const int* cols, float* X,
                                int64_t ldx, cudaStream_t st) {
    if (n <= 0 || s <= 0) return cudaSuccess;
    srtt_x_dense_kernel<<<blocks_for(n * s, 256), 256, 0, st>>>(n, s, dbits, cols, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_hrtt_table(uint64_t seed, int bits, uint16_t* tbl, cudaStream_t st) {
    if (bits > 15) return cudaErrorInvalidValue;     // entries hold c in 15 bits
    const int np = 1 << bits;
    hrtt_table_kernel<<<blocks_for(np, 256), 256, 0, st>>>(seed, bits, np, tbl);
    return cudaGetLastError();
}

// Rows j0 .. j0 + gridDim.x - 1 of the HRTT's X^T as BF16 bits: row j (over k < n,
// zero up to kpad) = d_k (H v_j)[k], v_j the signed indicator of bucket j (entries
// q = j + t s of the table).  One CTA per bucket: v_j scattered into shared memory
// (2^bits floats) and transformed in place by the unnormalised Walsh-Hadamard
// butterflies; the results are integers of magnitude at most the bucket size,
// exact in BF16 when that is at most 256.
__global__ void __launch_bounds__(1024) hrtt_xt_bf16_kernel(int64_t n, int64_t kpad, int s, int j0, int bits,
                                                            const uint32_t* __restrict__ dbits,
                                                            const uint16_t* __restrict__ tbl,
                                                            uint16_t* __restrict__ Xt, int64_t ldt, int planes,
                                                            int64_t plane_rows) {
    extern __shared__ float y[];
    const int N = 1 << bits, j = j0 + (int)blockIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) y[i] = 0.f;
    __syncthreads();
    for (int q = j + (int)threadIdx.x * s; q < N; q += (int)blockDim.x * s) {
        const uint32_t e = tbl[q];
        y[e & 0x7fffu] = (e >> 15) ? -1.f : 1.f;       // distinct coordinates: the table is a bijection
    }
    __syncthreads();
    for (int h = 1; h < N; h <<= 1) {
        for (int t = threadIdx.x; t < N / 2; t += blockDim.x) {
            const int i = (t / h) * 2 * h + (t % h);
            const float a = y[i], b = y[i + h];
            y[i] = a + b;
            y[i + h] = a - b;
        }
        __syncthreads();
    }
    uint16_t* row = Xt + (int64_t)blockIdx.x * ldt;
    uint16_t* row_lo = row + plane_rows * ldt;
    for (int64_t k = threadIdx.x; k < kpad; k += blockDim.x) {
        float v = 0.f;
        if (k < n) v = ((dbits[k >> 5] >> (k & 31)) & 1u) ? -y[k] : y[k];
        if (planes == 1) {
            row[k] = (uint16_t)(__float_as_uint(v) >> 16);
        } else {
            // an integer below 2^16 in magnitude: its nearest BF16 and the (exact,
            // at most 8-bit) remainder
            const uint32_t hb = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
            const float lo = v - __uint_as_float(hb << 16);
            row[k] = (uint16_t)hb;
            row_lo[k] = (uint16_t)(__float_as_uint(lo) >> 16);
        }
    }
}

cudaError_t launch_hrtt_xt_bf16(int64_t n, int64_t kpad, int s, int j0, int cnt, int bits, const uint32_t* dbits,
                                const uint16_t* tbl, uint16_t* Xt, int64_t ldt, cudaStream_t st, int planes,
                                int64_t plane_rows) {
    if (cnt <= 0) return cudaSuccess;
    if (bits < 0 || bits > 15 || s <= 0 || j0 < 0 || j0 + cnt > s || (planes != 1 && planes != 2) ||
        (planes == 2 && plane_rows < cnt))
        return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) << bits;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(hrtt_xt_bf16_kernel));
    if (e != cudaSuccess) return e;
    hrtt_xt_bf16_kernel<<<cnt, 1024, smem, st>>>(n, kpad, s, j0, bits, dbits, tbl, Xt, ldt, planes, plane_rows);
    return cudaGetLastError();
}

// Columns j0 .. j0+cnt-1 of the width-s hashed randomized DCT X (order N = 2^bits):
// X[k][j] = d_k sum over bucket j of sigma_c sqrt(2) w_c cos(pi (2k+1) c / 2N)
// (w_0 = 1/sqrt(2)).  The cosines come from the table cos(pi i / 2N), i in [0, N],
// held in shared memory, after the phase (2k+1) c is reduced modulo 4N in integers
// and folded onto [0, N].  Rows k and N-1-k take the same table entry: their
// phases differ by c (2N) - (2k+1) c, so their cosines differ by the sign (-1)^c.
// A thread forms both rows of one pair, each as an FP32 sum with a compensation
// term (Kahan), so the value is close to the correctly rounded sum.  Work items
// are (bucket, chunk of blockDim pairs), spread over a persistent grid; each
// item first stages its bucket as records (c, sigma_c sqrt(2) w_c, the same times
// (-1)^c) so the inner loop reads one 16-byte broadcast per entry.
// planes = 0: FP32 X row-major (X[k * ldx + j - j0], rows k < n); planes = 3: the
// three exact BF16 terms of the FP32 value as X^T planes (row j - j0 of plane t at
// Xt + (t * plane_rows + j - j0) * ldx, columns k < kpad, zeros for n <= k).
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ void hrct_store(int planes, float v, int64_t k, int jj, float* X, uint16_t* Xt,
                                           int64_t ldx, int64_t plane_rows) {
    if (planes == 0) {
        X[k * ldx + jj] = v;
    } else {
        uint32_t hi, mid, lo;
        tc::split3(v, 0.f, hi, mid, lo);       // the low halves hold the terms of v
        Xt[(int64_t)jj * ldx + k] = (uint16_t)(hi & 0xffffu);
        Xt[(plane_rows + jj) * ldx + k] = (uint16_t)(mid & 0xffffu);
        Xt[(2 * plane_rows + jj) * ldx + k] = (uint16_t)(lo & 0xffffu);
    }
}

__global__ void __launch_bounds__(512) hrct_x_kernel(int64_t n, int64_t kpad, int s, int j0, int cnt, int bits,
                                                     const uint32_t* __restrict__ dbits,
                                                     const uint16_t* __restrict__ tbl,
                                                     const float* __restrict__ ctab, int planes,
                                                     float* __restrict__ X, uint16_t* __restrict__ Xt, int64_t ldx,
                                                     int64_t plane_rows) {
    extern __shared__ __align__(16) float smf[];
    const int N = 1 << bits;
    // ceil(N / s) bucket records, then the N + 1 cosines with one padding word
    // after every 32 (cosine i at i + i / 32): within a branch of the fold the lanes
    // of a warp read indices 2c apart, and the padding spreads such power-of-two
    // multiples over the banks
    uint4* bucket = reinterpret_cast<uint4*>(smf);
    float* ct = smf + 4 * ((N + s - 1) / s);
    for (int i = threadIdx.x; i <= N; i += blockDim.x) ct[i + (i >> 5)] = ctab[i];
    const int64_t kend = planes == 0 ? n : kpad;
    const int kcov = (int)(kend < (int64_t)N ? kend : (int64_t)N);  // rows below N
    const int P = (N + 1) / 2 < kcov ? (N + 1) / 2 : kcov;           // pairs (k, N-1-k)
    const int chunks = (P + (int)blockDim.x - 1) / (int)blockDim.x;
    const int items = cnt * chunks;
    const uint32_t twoN = 2u * (uint32_t)N, fourN = 4u * (uint32_t)N, mask = fourN - 1u;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int jj = item / chunks, chunk = item - jj * chunks;
        const int j = j0 + jj;
        const int L = (N - j + s - 1) / s;                        // entries q = j + t s < N
        __syncthreads();                                          // the previous bucket is no longer read
        for (int t = threadIdx.x; t < L; t += blockDim.x) {
            const uint32_t e = tbl[j + t * s];
            const uint32_t c = e & 0x7fffu;
            float coef = c == 0 ? 1.f : 1.41421356237309515f;     // sqrt(2) w_c
            if (e >> 15) coef = -coef;                            // sigma_c
            const float coef_m = (c & 1u) ? -coef : coef;         // row N-1-k: times (-1)^c
            bucket[t] = make_uint4(c, __float_as_uint(coef), __float_as_uint(coef_m), 0u);
        }
        __syncthreads();
        const int p = chunk * (int)blockDim.x + (int)threadIdx.x;
        if (p >= P) continue;                                     // every thread runs the same items
        const int k = p, km = N - 1 - p;
        const bool vk = k < n, vm = km != k && km < n;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
        if (vk || vm) {
            const uint32_t odd = 2u * (uint32_t)k + 1u;           // < 2^16, c < 2^15: no overflow
            for (int t = 0; t < L; ++t) {
                const uint4 b = bucket[t];
                const uint32_t ph = (odd * b.x) & mask;
                const uint32_t ph2 = min(ph, fourN - ph);         // cos(2 pi - x) = cos x: [0, 2N]
                const uint32_t jx = min(ph2, twoN - ph2);         // cos(pi - x) = -cos x: [0, N]
                const float cv = ct[jx + (jx >> 5)];
                const bool neg = ph2 > (uint32_t)N;
                const float ca = __uint_as_float(b.y), cm = __uint_as_float(b.z);
                kahan_add(s0, c0, (neg ? -ca : ca) * cv);         // c = 0: ph = 0, cv = 1
                kahan_add(s1, c1, (neg ? -cm : cm) * cv);
            }
        }
        if (k < kend) {
            const float v = vk ? (((dbits[k >> 5] >> (k & 31)) & 1u) ? -s0 : s0) : 0.f;
            hrct_store(planes, v, k, jj, X, Xt, ldx, plane_rows);
        }
        if (km != k && km < kend) {
            const float v = vm ? (((dbits[km >> 5] >> (km & 31)) & 1u) ? -s1 : s1) : 0.f;
            hrct_store(planes, v, km, jj, X, Xt, ldx, plane_rows);
        }
    }
    // rows N .. kend-1 (a padded X^T wider than the order): zeros
    const int64_t extra = kend > (int64_t)N ? kend - N : 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < extra * cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        hrct_store(planes, 0.f, N + i % extra, (int)(i / extra), X, Xt, ldx, plane_rows);
}

cudaError_t launch_hrct_x(int64_t n, int64_t kpad, int s, int j0, int cnt, int bits, const uint32_t* dbits,
                          const uint16_t* tbl, const float* ctab, int planes, float* X, uint16_t* Xt, int64_t ldx,
                          int64_t plane_rows, cudaStream_t st) {
    if (cnt <= 0) return cudaSuccess;
    if (bits < 0 || bits > 15 || s <= 0 || j0 < 0 || j0 + cnt > s || n <= 0 || n > (int64_t(1) << bits) ||
        (planes != 0 && planes != 3) || (planes == 0 && ldx < cnt) || (planes == 3 && (plane_rows < cnt || kpad < n ||
        ldx < kpad)))
        return cudaErrorInvalidValue;
    const int N = 1 << bits;
    const size_t smem = sizeof(float) * (size_t)(N + 1 + (N >> 5) + 1) + sizeof(uint4) * (size_t)((N + s - 1) / s);
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(hrct_x_kernel));
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hrct_x_kernel, 512, smem);
    if (e != cudaSuccess) return e;
    const int64_t kend = planes == 0 ? n : kpad;
    const int64_t P = std::min<int64_t>((N + 1) / 2, std::min<int64_t>(kend, N));
    const int64_t items = (int64_t)cnt * ((P + 511) / 512);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)sms * std::max(per_sm, 1)));
    hrct_x_kernel<<<grid, 512, smem, st>>>(n, kpad, s, j0, cnt, bits, dbits, tbl, ctab, planes, X, Xt, ldx,
                                           plane_rows);
    return cudaGetLastError();
}

cudaError_t launch_hrtt_x_dense(int64_t n, int s, int bits, const uint32_t* dbits, const uint16_t* tbl,
                                float* X, int64_t ldx, cudaStream_t st) {
    if (n <= 0 || s <= 0) return cudaSuccess;
    hrtt_x_dense_kernel<<<blocks_for(n * s, 256), 256, 0, st>>>(n, s, 1 << bits, dbits, tbl, X, ldx);
    return cudaGetLastError();
}

cudaError_t launch_srtt_y_dense(int64_t m, int r2, const uint32_t* dbits, const int* rows, float* Y,
                                int64_t ldy, cudaStream_t st) {
    if (m <= 0 || r2 <= 0) return cudaSuccess;
    srtt_y_dense_kernel<<<blocks_for(m * r2, 256), 256, 0, st>>>(m, r2, dbits, rows, Y, ldy);
    return cudaGetLastError();
}

namespace {
__global__ void cos_table_kernel(int nbits, float* __restrict__ ctab) {
    const int64_t N = int64_t(1) << nbits;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= N; j += (int64_t)gridDim.x * blockDim.x)
        ctab[j] = (float)cospi((double)j / (double)(2 * N));   // j / 2N is exact in FP64
}
}  // namespace

cudaError_t launch_cos_table(int nbits, float* ctab, cudaStream_t st) {
    if (nbits < 0 || nbits > 31) return cudaErrorInvalidValue;
    const int64_t N = int64_t(1) << nbits;
    const int blocks = (int)std::min<int64_t>((N + 256) / 256, 4096);
    cos_table_kernel<<<blocks, 256, 0, st>>>(nbits, ctab);
    return cudaGetLastError();
}

}  // namespace re
