// Device helpers shared by the CUDA translation units of librankest.
//
// The counter-based generator below draws the random embeddings X and Y of the
// two-sided sketch (Algorithm 1 steps 2 and 5; Gaussian embeddings G/sqrt(r) in
// the Sec. 1 notation; SRTT signs and row sampling of Eq. (Theta)).  It follows
// this written specification, which the CPU oracle implements independently:
//
//  * Philox4x32-10 (Salmon et al., SC'11): counter (c0,c1,c2,c3), key
//    (seed lo, seed hi); round (hi0,lo0)=mulhilo(0xD2511F53,c0),
//    (hi1,lo1)=mulhilo(0xCD9E8D57,c2), c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0);
//    key += (0x9E3779B9, 0xBB67AE85) between rounds; 10 rounds.
//  * Box-Muller in binary32, every operation correctly rounded, no FMA
//    contraction (hence the __f*_rn intrinsics): u1 = ((a>>8)+1) 2^-24,
//    u2 = (b>>8) 2^-24, r = sqrt(-2 ln u1), angle 2 pi u2 split into a quadrant
//    and theta in [0, pi/2); ln by the atanh series after reducing the mantissa
//    to [sqrt(1/2), sqrt(2)), sin/cos by Taylor polynomials (own code, not a
//    libm); result rounded to BF16 (nearest even) and then to the nearest
//    multiple of 2^-13 (ties to even; zero is +0).  Values of magnitude >= 2^-6
//    are BF16 multiples of 2^-13 already, so the second rounding moves only values
//    below 2^-6, by at most 2^-14; every normal is then an integer multiple of
//    2^-13 below 6 in magnitude (16-bit fixed point, exact in BF16 and FP16), which
//    splits exactly into two 8-bit pieces on the grids 2^-5 and 2^-13.
//  * X(k, j) = normal (j mod 4) of Philox(k, j/4, 1, 0); Y(q, i) = normal (q mod 4)
//    of Philox(i, q/4, 2, 0); SRTT sign d_j = bit (j mod 128) of
//    Philox(j/128, 0, stream, 0) (stream 3 right, 5 left); sampled index
//    pi(k) from a 4-round Feistel bijection of [0, 2^b) whose round function is
//    word 0 of Philox(half, round, stream, 0) (stream 4 right, 6 left).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace re {

// Lets `kern` take as much dynamic shared memory as the device allows beside its
// static shared memory.  The limit is one fixed value per kernel, so host threads
// that launch the same kernel with different sizes cannot lower it under one
// another's launches; a launch still reserves only the size it requests.
inline cudaError_t allow_dynamic_smem(const void* kern) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    int optin = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

constexpr uint32_t kStreamGX = 1;
constexpr uint32_t kStreamGY = 2;
constexpr uint32_t kStreamDX = 3;
constexpr uint32_t kStreamPX = 4;
constexpr uint32_t kStreamDY = 5;
constexpr uint32_t kStreamPY = 6;
constexpr uint32_t kStreamSX = 7;   // CountSketch signs of the HRTT (one per transform coordinate)

struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = mulhi32(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = mulhi32(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// ---- binary32 transform (device only; correctly rounded intrinsics) ----------
#ifdef __CUDACC__
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }

__device__ __forceinline__ float ln_pos(float u) {
    const uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float f = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (f > 0x1.6a09e6p+0f) {
        f = fmul(f, 0.5f);
        e += 1;
    }
    const float t = __fdiv_rn(fsub(f, 1.0f), fadd(f, 1.0f));
    const float t2 = fmul(t, t);
    float p = 0x1.745d18p-4f;                 // 1/11
    p = fadd(fmul(p, t2), 0x1.c71c72p-4f);    // 1/9
    p = fadd(fmul(p, t2), 0x1.24924ap-3f);    // 1/7
    p = fadd(fmul(p, t2), 0x1.99999ap-3f);    // 1/5
    p = fadd(fmul(p, t2), 0x1.555556p-2f);    // 1/3
    p = fadd(fmul(p, t2), 1.0f);
    const float lnf = fmul(fmul(2.0f, t), p);
    return fadd(fmul((float)e, 0x1.62e430p-1f), lnf);
}

__device__ __forceinline__ void sincos_quarter(float th, float& s, float& c) {
    const float t2 = fmul(th, th);
    float ps = 0x1.612462p-33f;               // 1/13!
    ps = fadd(fmul(ps, t2), -0x1.ae6456p-26f);
    ps = fadd(fmul(ps, t2), 0x1.71de3ap-19f);
    ps = fadd(fmul(ps, t2), -0x1.a01a02p-13f);
    ps = fadd(fmul(ps, t2), 0x1.111112p-7f);
    ps = fadd(fmul(ps, t2), -0x1.555556p-3f);
    ps = fmul(ps, t2);
    s = fadd(fmul(th, ps), th);
    float pc = -0x1.93974ap-37f;              // -1/14!
    pc = fadd(fmul(pc, t2), 0x1.1eed8ep-29f);
    pc = fadd(fmul(pc, t2), -0x1.27e4fcp-22f);
    pc = fadd(fmul(pc, t2), 0x1.a01a02p-16f);
    pc = fadd(fmul(pc, t2), -0x1.6c16c2p-10f);
    pc = fadd(fmul(pc, t2), 0x1.555556p-5f);
    pc = fadd(fmul(pc, t2), -0.5f);
    c = fadd(fmul(pc, t2), 1.0f);
}

__device__ __forceinline__ float round_normal(float z) {
    uint32_t b = __float_as_uint(z);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    const float r = __uint_as_float(b);
    if (fabsf(r) >= 0x1p-6f) return r;
    // |r| < 2^-6: 1536 + r lies in [1024, 2048), whose spacing is 2^-13, so the sum
    // rounds r to the 2^-13 grid (ties to even) and the difference is exact (+0 for 0)
    return __fsub_rn(__fadd_rn(r, 1536.0f), 1536.0f);
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
    const float u1 = fmul(fadd((float)(a >> 8), 1.0f), 0x1p-24f);
    const float u2 = fmul((float)(b >> 8), 0x1p-24f);
    const float r = __fsqrt_rn(fmul(-2.0f, ln_pos(u1)));
    const float v = fmul(u2, 4.0f);
    const int q = (int)v;
    const float fr = fsub(v, (float)q);
    const float th = fmul(fr, 0x1.921fb6p+0f);
    float s, c;
    sincos_quarter(th, s, c);
    float cp, sp;
    if (q == 0) {
        cp = c; sp = s;
    } else if (q == 1) {
        cp = -s; sp = c;
    } else if (q == 2) {
        cp = -c; sp = -s;
    } else {
        cp = s; sp = -c;
    }
    z0 = round_normal(fmul(r, cp));
    z1 = round_normal(fmul(r, sp));
}

// The four normals of Philox((c0, c1, stream, 0)).
__device__ __forceinline__ void normals4(uint32_t c0, uint32_t c1, uint32_t stream, uint64_t seed,
                                         float z[4]) {
    const U4 w = philox(c0, c1, stream, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
    box_muller(w.x, w.y, z[0], z[1]);
    box_muller(w.z, w.w, z[2], z[3]);
}
#endif  // __CUDACC__

// Keyed Feistel bijection of [0, 2^bits) (host and device).
__host__ __device__ __forceinline__ uint32_t feistel(uint32_t x, int bits, uint32_t stream,
                                                     uint64_t seed) {
    if (bits == 0) return 0u;
    int wlo = bits >> 1;
    int whi = bits - wlo;
    uint32_t lo = x & ((1u << wlo) - 1u);
    uint32_t hi = x >> wlo;
    for (uint32_t r = 0; r < 4; ++r) {
        const uint32_t f = philox(hi, r, stream, 0u, (uint32_t)seed, (uint32_t)(seed >> 32)).x;
        const uint32_t nlo = hi;
        const uint32_t nhi = lo ^ (f & ((1u << wlo) - 1u));
        lo = nlo;
        hi = nhi;
        const int t = wlo;
        wlo = whi;
        whi = t;
    }
    return (hi << wlo) | lo;
}

__host__ __device__ __forceinline__ int pow2_bits(int64_t n) {
    int b = 0;
    while ((int64_t(1) << b) < n) ++b;
    return b;
}

}  // namespace re
