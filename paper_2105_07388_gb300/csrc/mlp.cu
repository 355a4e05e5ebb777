// Sketch-size proposal network: a small MLP that, from the sketched singular
// values of a cheap first sketch (s = 16), predicts the ladder width at which
// Algorithm 1's read-off will succeed, so the estimator can append straight to
// that width instead of doubling (the paper's closing discussion, Sec. 7, asks
// for choosing a new r1 from the information of the first run).  Every
// prediction is still verified by the plain criterion on the nested leading
// blocks of the core, which is also the fallback.
//
//   x (18) -> h1 = relu(W1 x + b1) (128) -> h2 = relu(W2 h1 + b2) (128)
//          -> z = W3 h2 + b3 (12 logits), class c <-> width 8 * 2^c.
//
// Weights are used in BF16 (rounded from FP32 master copies after every update)
// with FP32 accumulation; biases stay FP32.  Forward: one CTA of 128 threads per
// sample.  Backward: softmax cross-entropy averaged over the batch, per-sample
// contributions accumulated with atomics into FP32 gradients.  Optimiser: Adam.
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

constexpr int kIn = kMlpIn, kH = kMlpHidden, kOut = kMlpOut;
// parameter offsets (floats) in the flat vector: W1 b1 W2 b2 W3 b3
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kParams = oB3 + kOut;
static_assert(kParams == kMlpParams, "parameter count");

__device__ __forceinline__ float bf16r(float x) {
    uint32_t b = __float_as_uint(x);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    return __uint_as_float(b);
}

// Forward for one sample per CTA; stores h1, h2, z when keep != nullptr.
__global__ void __launch_bounds__(kH) mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                         int count, float* __restrict__ logits,
                                                         float* __restrict__ keep) {
    __shared__ float x[kIn], h1[kH], h2[kH];
    const int b = blockIdx.x, t = threadIdx.x;
    if (b >= count) return;
    if (t < kIn) x[t] = X[(int64_t)b * kIn + t];
    __syncthreads();
    float a = P[oB1 + t];
    for (int k = 0; k < kIn; ++k) a = fmaf(bf16r(P[oW1 + t * kIn + k]), x[k], a);
    h1[t] = fmaxf(a, 0.f);
    __syncthreads();
    a = P[oB2 + t];
    for (int k = 0; k < kH; ++k) a = fmaf(bf16r(P[oW2 + t * kH + k]), h1[k], a);
    h2[t] = fmaxf(a, 0.f);
    __syncthreads();
    if (t < kOut) {
        a = P[oB3 + t];
        for (int k = 0; k < kH; ++k) a = fmaf(bf16r(P[oW3 + t * kH + k]), h2[k], a);
        logits[(int64_t)b * kOut + t] = a;
    }
    if (keep) {
        float* kp = keep + (int64_t)b * (2 * kH);
        kp[t] = h1[t];
        kp[kH + t] = h2[t];
    }
}

// Backward of the mean softmax cross-entropy; adds this sample's gradient / count into G.
__global__ void __launch_bounds__(kH) mlp_backward_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                          const int* __restrict__ y, int count,
                                                          const float* __restrict__ logits,
                                                          const float* __restrict__ keep, float* __restrict__ G,
                                                          float* __restrict__ loss) {
    __shared__ float x[kIn], h1[kH], h2[kH], dz[kOut], dh2[kH];
    const int b = blockIdx.x, t = threadIdx.x;
    if (b >= count) return;
    const float inv = 1.f / (float)count;
    if (t < kIn) x[t] = X[(int64_t)b * kIn + t];
    h1[t] = keep[(int64_t)b * 2 * kH + t];
    h2[t] = keep[(int64_t)b * 2 * kH + kH + t];
    if (t == 0) {
        const float* z = logits + (int64_t)b * kOut;
        float mx = z[0];
        for (int c = 1; c < kOut; ++c) mx = fmaxf(mx, z[c]);
        float se = 0.f;
        for (int c = 0; c < kOut; ++c) se += expf(z[c] - mx);
        const int lab = y[b];
        for (int c = 0; c < kOut; ++c) dz[c] = (expf(z[c] - mx) / se - (c == lab ? 1.f : 0.f)) * inv;
        atomicAdd(loss, (logf(se) + mx - z[lab]) * inv);
    }
    __syncthreads();
    // layer 3
    if (t < kOut) atomicAdd(&G[oB3 + t], dz[t]);
    for (int c = 0; c < kOut; ++c) atomicAdd(&G[oW3 + c * kH + t], dz[c] * h2[t]);
    float g = 0.f;
    for (int c = 0; c < kOut; ++c) g = fmaf(bf16r(P[oW3 + c * kH + t]), dz[c], g);
    dh2[t] = h2[t] > 0.f ? g : 0.f;
    __syncthreads();
    // layer 2: row t of W2
    atomicAdd(&G[oB2 + t], dh2[t]);
    for (int k = 0; k < kH; ++k) atomicAdd(&G[oW2 + t * kH + k], dh2[t] * h1[k]);
    g = 0.f;
    for (int j = 0; j < kH; ++j) g = fmaf(bf16r(P[oW2 + j * kH + t]), dh2[j], g);
    const float dh1 = h1[t] > 0.f ? g : 0.f;
    // layer 1: row t of W1
    atomicAdd(&G[oB1 + t], dh1);
    for (int k = 0; k < kIn; ++k) atomicAdd(&G[oW1 + t * kIn + k], dh1 * x[k]);
}

__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float wd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float g = G[i] + wd * P[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void argmax_kernel(const float* __restrict__ logits, int count, int* __restrict__ cls) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count) return;
    const float* z = logits + (int64_t)b * kOut;
    int best = 0;
    for (int c = 1; c < kOut; ++c)
        if (z[c] > z[best]) best = c;
    cls[b] = best;
}

// Features of one estimate from the s = 16 sketched singular values (scaled,
// descending): 14 trusted values as log10(sigma_i / (eps sigma_1)), log10 of
// the oriented rows and columns, log10(1/eps), and the mean log10 decay per
// index over the last seven trusted values.
__global__ void features_kernel(const double* __restrict__ sigma16, double eps, int64_t rows, int64_t cols,
                                float* __restrict__ f) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double s1 = sigma16[0] > 0.0 ? sigma16[0] : 1e-300;
    for (int i = 0; i < 14; ++i) {
        const double v = fmax(sigma16[i], 1e-30 * s1);
        f[i] = (float)log10(v / (eps * s1));
    }
    f[14] = (float)log10((double)rows);
    f[15] = (float)log10((double)cols);
    f[16] = (float)log10(1.0 / eps);
    f[17] = (f[13] - f[7]) / 6.f;
}

}  // namespace

cudaError_t mlp_forward(const float* P, const float* X, int count, float* logits, float* keep, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    mlp_forward_kernel<<<count, kH, 0, st>>>(P, X, count, logits, keep);
    return cudaGetLastError();
}

cudaError_t mlp_backward(const float* P, const float* X, const int* y, int count, const float* logits,
                         const float* keep, float* G, float* loss, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    mlp_backward_kernel<<<count, kH, 0, st>>>(P, X, y, count, logits, keep, G, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* P, const float* G, float* M, float* V, float lr, int step, float wd, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(P, G, M, V, kParams, lr, b1, b2, 1e-8f, c1, c2, wd);
    return cudaGetLastError();
}

cudaError_t mlp_argmax(const float* logits, int count, int* cls, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    argmax_kernel<<<(count + 127) / 128, 128, 0, st>>>(logits, count, cls);
    return cudaGetLastError();
}

cudaError_t mlp_features(const double* sigma16, double eps, int64_t rows, int64_t cols, float* f, cudaStream_t st) {
    features_kernel<<<1, 32, 0, st>>>(sigma16, eps, rows, cols, f);
    return cudaGetLastError();
}

// Deterministic initialisation (He-uniform from a counter hash), host side.
void mlp_init_host(float* P, uint64_t seed) {
    auto u01 = [&](uint32_t i) {
        const U4 w = philox(i, 0u, 7u, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        return ((w.x >> 8) + 0.5f) * (1.0f / 16777216.0f);
    };
    std::memset(P, 0, sizeof(float) * kParams);
    const float a1 = sqrtf(6.f / kIn), a2 = sqrtf(6.f / kH), a3 = sqrtf(6.f / kH);
    for (int i = 0; i < kH * kIn; ++i) P[oW1 + i] = (2.f * u01(oW1 + i) - 1.f) * a1;
    for (int i = 0; i < kH * kH; ++i) P[oW2 + i] = (2.f * u01(oW2 + i) - 1.f) * a2;
    for (int i = 0; i < kOut * kH; ++i) P[oW3 + i] = (2.f * u01(oW3 + i) - 1.f) * a3;
}

}  // namespace re
