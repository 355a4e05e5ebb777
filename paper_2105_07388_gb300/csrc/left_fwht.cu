// Left sketch with a subsampled randomized Hadamard Theta = S H D (Eq. (Theta) of
// Sec. 4, Y unscaled: entries d_i H[pi_Y(q), i]) at the O(m s log m) cost the
// paper quotes for it (Sec. 4; Sec. 5.1 on the rank-estimation overhead): every
// column of D (A X) is transformed once by a fast Walsh-Hadamard transform over
// the zero-padded m_pad = 2^b rows and kept, Z = H D AX (m_pad x s, row-major);
// core entry (q, c) is then the sampled coordinate Z[pi_Y(q), c].  Appending
// columns of X transforms only the new columns; appending rows of Y only samples
// more rows of Z.
//
// The transform runs in passes over groups of at most kMaxBits index bits: a CTA
// takes the 2^nb rows i = base + t 2^lo (t < 2^nb; base fixes every other bit)
// of a chunk of kCW columns into shared memory, applies the nb butterfly stages
// and writes them back.  The first pass reads d_i AX[i, c] (zero for i >= m).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kCW = 16;        // columns per CTA
constexpr int kMaxBits = 10;   // index bits per pass: 1024 x 16 floats = 64 KB of shared memory
constexpr int kPassThreads = 256;

template <bool FIRST>
__global__ void __launch_bounds__(kPassThreads) fwht_rows_pass_kernel(const float* __restrict__ AX, int64_t ldax,
                                                                      int64_t M, const uint32_t* __restrict__ dbits,
                                                                      float* __restrict__ Z, int64_t ldz, int lo,
                                                                      int nb, int c0, int nc) {
    extern __shared__ float tile[];                   // (1 << nb) rows x kCW columns
    const int L = 1 << nb;
    const int64_t other = blockIdx.x;                 // the bits outside [lo, lo + nb)
    const int64_t base = (other & ((int64_t(1) << lo) - 1)) | ((other >> lo) << (lo + nb));
    const int64_t stride = int64_t(1) << lo;
    const int cbeg = c0 + (int)blockIdx.y * kCW;
    const int cw = min(kCW, c0 + nc - cbeg);
    for (int e = threadIdx.x; e < L * kCW; e += blockDim.x) {
        const int t = e / kCW, c = e % kCW;
        const int64_t i = base + (int64_t)t * stride;
        float v = 0.0f;
        if (c < cw) {
            if constexpr (FIRST) {
                if (i < M) {
                    v = AX[i * ldax + cbeg + c];
                    if ((dbits[i >> 5] >> (i & 31)) & 1u) v = -v;
                }
            } else {
                v = Z[i * ldz + cbeg + c];
            }
        }
        tile[e] = v;
    }
    __syncthreads();
    for (int h = 1; h < L; h <<= 1) {
        for (int e = threadIdx.x; e < (L / 2) * kCW; e += blockDim.x) {
            const int b = e / kCW, c = e % kCW;
            const int t0 = (b / h) * 2 * h + (b % h);
            const float x = tile[t0 * kCW + c], y = tile[(t0 + h) * kCW + c];
            tile[t0 * kCW + c] = x + y;
            tile[(t0 + h) * kCW + c] = x - y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < L * kCW; e += blockDim.x) {
        const int t = e / kCW, c = e % kCW;
        if (c < cw) Z[(base + (int64_t)t * stride) * ldz + cbeg + c] = tile[e];
    }
}

__global__ void sample_core_kernel(const float* __restrict__ Z, int64_t ldz, const int* __restrict__ perm, int row0,
                                   int R, int col0, int S, double* __restrict__ core, int64_t ld_core) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * S) return;
    const int r = (int)(idx / S), c = (int)(idx % S);
    core[(int64_t)(row0 + r) * ld_core + col0 + c] = (double)Z[(int64_t)perm[row0 + r] * ldz + col0 + c];
}

}  // namespace

cudaError_t launch_left_srtt_transform(const float* AX, int64_t ldax, int64_t M, int mbits, const uint32_t* dbits,
                                       int c0, int c1, float* Z, int64_t ldz, cudaStream_t st) {
    if (c1 <= c0 || M <= 0) return cudaSuccess;
    if (mbits > 31 || ldz < c1) return cudaErrorInvalidValue;
    const int nc = c1 - c0;
    const unsigned gy = (unsigned)((nc + kCW - 1) / kCW);
    const int smem_max = (int)(sizeof(float) * ((size_t)kCW << kMaxBits));   // 64 KB: above the default 48 KB
    cudaError_t ea = allow_dynamic_smem(reinterpret_cast<const void*>(fwht_rows_pass_kernel<true>));
    if (ea == cudaSuccess)
        ea = allow_dynamic_smem(reinterpret_cast<const void*>(fwht_rows_pass_kernel<false>));
    if (ea != cudaSuccess) return ea;
    int lo = 0;
    bool first = true;
    do {
        const int nb = std::min(kMaxBits, mbits - lo);
        const size_t smem = sizeof(float) * ((size_t)kCW << nb);
        const dim3 grid((unsigned)(int64_t(1) << (mbits - nb)), gy);
        if (first) {
            fwht_rows_pass_kernel<true><<<grid, kPassThreads, smem, st>>>(AX, ldax, M, dbits, Z, ldz, lo, nb, c0, nc);
        } else {
            fwht_rows_pass_kernel<false><<<grid, kPassThreads, smem, st>>>(AX, ldax, M, dbits, Z, ldz, lo, nb, c0, nc);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        lo += nb;
        first = false;
    } while (lo < mbits);
    return cudaSuccess;
}

cudaError_t launch_left_srtt_sample(const float* Z, int64_t ldz, const int* perm, int row0, int R, int col0, int S,
                                    double* core, int64_t ld_core, cudaStream_t st) {
    const int64_t total = (int64_t)R * S;
    if (total <= 0) return cudaSuccess;
    sample_core_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Z, ldz, perm, row0, R, col0, S, core,
                                                                        ld_core);
    return cudaGetLastError();
}

}  // namespace re
