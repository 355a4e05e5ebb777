// Right sketch with a subsampled randomized Hadamard transform (Sec. 3.4, SRTT;
// Eq. (Theta) of Sec. 4 applied from the right: X = D H S^T over the dimension
// n_pad = 2^ceil(log2 n) with A zero padded, Sec. 4 on zero padding):
//
//     AX[r, k] = sum_j A[r, j] d_j H[j, pi(k)],   H[j, c] = (-1)^popcount(j & c).
//
// Each row is transformed by a fast Walsh-Hadamard transform (O(n log n) per
// row, the cost quoted for SRTTs in Sec. 3.4) and the s sampled outputs are
// gathered.  A row of 2^L values is held by T = 2^floor(L/2) threads with
// E = 2^L / T values each in registers:
//   phase A  coalesced load, index = r*T + j (thread j, register r); the
//            butterflies over the register index cover bits [log T, L);
//   transpose through shared memory with an XOR swizzle (conflict-free both ways);
//   phase B  index = j*E + r; butterflies over register offsets < T cover bits
//            [0, log T);
//   gather   the sampled outputs pi(k) from shared memory.
// Because H_{2N}[i, c] = H_N[i, c] for i, c < N and padded inputs are zero, a
// transform longer than n_pad gives the same sampled values, so four kernel
// sizes (2^8, 2^10, 2^12, 2^14) serve every n <= 16384.  Longer rows
// (n <= 32768) use a shared-memory-only transform, one row per CTA.
//
// The same kernels give the hashed transform (HRTT, Sec. 3.4: the sampling S
// replaced by a CountSketch C): instead of gathering s sampled coordinates,
// output k adds every coordinate c of its bucket with the sign sigma_c.  The
// buckets come from one table of n_pad 16-bit entries (entry q = pi(q) with
// the sign in bit 15; bucket k = entries q = k mod s), so a row costs n_pad
// extra shared-memory reads on top of the transform.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tc_common.cuh"

namespace re {

namespace {

template <typename TA>
__device__ __forceinline__ float load_oriented(const TA* A, int64_t lda, int64_t r, int64_t c,
                                               bool trans) {
    return trans ? (float)__ldg(A + c * lda + r) : (float)__ldg(A + r * lda + c);
}

template <int E, int H_LIMIT>
__device__ __forceinline__ void fwht_regs(float (&x)[E]) {
#pragma unroll
    for (int h = 1; h < H_LIMIT; h <<= 1) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if ((r & h) == 0) {
                const float a = x[r], b = x[r + h];
                x[r] = a + b;
                x[r + h] = a - b;
            }
        }
    }
}

// HRTT outputs of one transformed row y (y[phys(c)] = coordinate c), any s:
// output k adds the entries q = k, k + s, ... < np of the table in that order.
// Thread j of T makes outputs j, j + T, ...
template <typename Phys>
__device__ __forceinline__ void hashed_outputs_any(const float* y, Phys phys, const uint16_t* __restrict__ htab,
                                                   int np, int s, int j, int T, float* __restrict__ out) {
    for (int k = j; k < s; k += T) {
        float acc = 0.0f;
        for (int q = k; q < np; q += s) {
            const uint32_t e = __ldg(htab + q);
            const float v = y[phys((int)(e & 0x7fffu))];
            acc += (e & 0x8000u) ? -v : v;
        }
        out[k] = acc;
    }
}

template <int LOGN, bool TRANS, typename TA>
__global__ void __launch_bounds__(128) srht_reg_kernel(const TA* __restrict__ A, int64_t lda,
                                                       int64_t M, int64_t N,
                                                       const uint32_t* __restrict__ dbits,
                                                       const int* __restrict__ cols,
                                                       const uint16_t* __restrict__ htab, int hnp, int s,
                                                       float* __restrict__ C, int64_t ldc) {
    constexpr int NP = 1 << LOGN;
    constexpr int LOGT = LOGN / 2;
    constexpr int T = 1 << LOGT;
    constexpr int LOGE = LOGN - LOGT;
    constexpr int E = 1 << LOGE;
    constexpr int G = 128 / T;                        // rows per CTA iteration
    constexpr int PITCH = NP + (T < 32 ? 16 : 0);
    constexpr int XMASK = (E < 32 ? E : 32) - 1;
    extern __shared__ float4 smem4[];
    float* buf = reinterpret_cast<float*>(smem4);     // G x PITCH
    uint32_t* sd = reinterpret_cast<uint32_t*>(buf + G * PITCH);
    int* scol = reinterpret_cast<int*>(sd + NP / 32);

    const int64_t nwords = (N + 31) / 32;
    for (int w = threadIdx.x; w < NP / 32; w += blockDim.x) sd[w] = (w < nwords) ? dbits[w] : 0u;
    if (!htab)
        for (int k = threadIdx.x; k < s; k += blockDim.x) scol[k] = cols[k];
    __syncthreads();

    const int g = threadIdx.x / T;
    const int j = threadIdx.x % T;
    float* gb = buf + g * PITCH;
    auto phys = [](int idx) { return idx ^ ((idx >> LOGE) & XMASK); };

    for (int64_t row0 = (int64_t)blockIdx.x * G; row0 < M; row0 += (int64_t)gridDim.x * G) {
        const int64_t row = row0 + g;
        const bool live = row < M;
        float x[E];
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const int idx = r * T + j;
            float v = 0.0f;
            if (live && idx < N) {
                v = load_oriented(A, lda, row, idx, TRANS);
                if ((sd[idx >> 5] >> (idx & 31)) & 1u) v = -v;
            }
            x[r] = v;
        }
        fwht_regs<E, E>(x);
#pragma unroll
        for (int r = 0; r < E; ++r) gb[phys(r * T + j)] = x[r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < E; ++r) x[r] = gb[phys(j * E + r)];
        __syncthreads();
        fwht_regs<E, T>(x);
#pragma unroll
        for (int r = 0; r < E; ++r) gb[phys(j * E + r)] = x[r];
        __syncthreads();
        if (live) {
            if (htab)
                hashed_outputs_any(gb, phys, htab, hnp, s, j, T, C + row * ldc);
            else
                for (int k = j; k < s; k += T) C[row * ldc + k] = gb[phys(scol[k])];
        }
        __syncthreads();
    }
}

// Rows longer than 2^14: whole row in shared memory, radix-2 stages.
template <bool TRANS, typename TA>
__global__ void __launch_bounds__(1024) srht_smem_kernel(const TA* __restrict__ A, int64_t lda,
                                                         int64_t M, int64_t N, int logn,
                                                         const uint32_t* __restrict__ dbits,
                                                         const int* __restrict__ cols,
                                                         const uint16_t* __restrict__ htab, int s,
                                                         float* __restrict__ C, int64_t ldc) {
    extern __shared__ float4 smem4[];
    float* buf = reinterpret_cast<float*>(smem4);
    const int np = 1 << logn;
    for (int64_t row = blockIdx.x; row < M; row += gridDim.x) {
        for (int idx = threadIdx.x; idx < np; idx += blockDim.x) {
            float v = 0.0f;
            if (idx < N) {
                v = load_oriented(A, lda, row, idx, TRANS);
                if ((__ldg(dbits + (idx >> 5)) >> (idx & 31)) & 1u) v = -v;
            }
            buf[idx] = v;
        }
        __syncthreads();
        for (int h = 1; h < np; h <<= 1) {
            for (int b = threadIdx.x; b < np / 2; b += blockDim.x) {
                const int lo = (b / h) * 2 * h + (b % h);
                const float a = buf[lo], c = buf[lo + h];
                buf[lo] = a + c;
                buf[lo + h] = a - c;
            }
            __syncthreads();
        }
        if (htab)
            hashed_outputs_any(buf, [](int c) { return c; }, htab, np, s, (int)threadIdx.x, (int)blockDim.x,
                               C + row * ldc);
        else
            for (int k = threadIdx.x; k < s; k += blockDim.x) C[row * ldc + k] = buf[cols[k]];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP32 rows with n_pad = 2^L, L = 12..14, aligned and not transposed: T = 2^(L-5)
// threads per row, 32 values per thread, three register phases joined by two
// shared-memory transposes (logical index bits in registers per phase):
//   phase 1  bits {0, 1} and [L-3, L): coalesced float4 loads, r*4T + 4j + q
//   phase 2  bits [2, 7):  thread = (idx >> 7, idx & 3)
//   phase 3  bits [7, L-3) of the register bits [7, 12): thread = (idx >> 12, idx & 127)
// Shared memory holds the row with its 16-byte chunks XOR-swizzled inside each
// 512-byte block by the block index, which makes the float4 stores of phase 1
// and the scalar loads and stores of phases 2 and 3 conflict-free.  Butterflies
// on register bits 1..4 run two at a time with packed FP32x2 add/sub (round to
// nearest, as scalar); bit 0 pairs neighbours and stays scalar.
__device__ __forceinline__ int phys_sw(int idx) {
    const int B = idx >> 7;
    return (B << 7) | ((((idx >> 2) & 31) ^ (B & 7)) << 2) | (idx & 3);
}

// phys_sw in closed form for the two transposes of thread j: phase 2 touches
// logical base + 4c (base = (j >> 2) 128 + (j & 3)), at o2[c & 7] + 4 (c & 24);
// phase 3 touches logical (j >> 7) 4096 + (j & 127) + 128 k, at o3[k & 7] + 128 k.
// With c and k unrolled, every access is a precomputed register plus an
// immediate offset.
__device__ __forceinline__ void sw_offsets(int j, int (&o2)[8], int (&o3)[8]) {
    const int b = (j >> 2) & 7, p2 = (j >> 2) * 128 + (j & 3);
    const int jj = (j & 127) >> 2, p3 = (j >> 7) * 4096 + (j & 3);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        o2[q] = p2 + 4 * (q ^ b);
        o3[q] = p3 + 4 * (jj ^ q);
    }
}

__device__ __forceinline__ void bfly2(float& a0, float& a1, float& b0, float& b1) {
    unsigned long long A, B, S, D;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a0), "f"(a1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b0), "f"(b1));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(S) : "l"(A), "l"(B));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(D) : "l"(A), "l"(B));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(S));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(b0), "=f"(b1) : "l"(D));
}

// butterflies over register-index bit H (a power of two) of 32 values
template <int H>
__device__ __forceinline__ void stage32(float (&x)[32]) {
    if constexpr (H == 1) {
        // neighbours x[r], x[r+1] are not a packed pair of the next stages' layout:
        // scalar butterflies here avoid moving registers in and out of pairs
#pragma unroll
        for (int r = 0; r < 32; r += 2) {
            const float a = x[r], b = x[r + 1];
            x[r] = a + b;
            x[r + 1] = a - b;
        }
    } else {
#pragma unroll
        for (int r = 0; r < 32; r += 2)
            if ((r & H) == 0) bfly2(x[r], x[r + 1], x[r + H], x[r + H + 1]);
    }
}

template <int NB>   // the first NB register-index bits
__device__ __forceinline__ void fwht32(float (&x)[32]) {
    if constexpr (NB > 0) stage32<1>(x);
    if constexpr (NB > 1) stage32<2>(x);
    if constexpr (NB > 2) stage32<4>(x);
    if constexpr (NB > 3) stage32<8>(x);
    if constexpr (NB > 4) stage32<16>(x);
}

template <int L>
__global__ void __launch_bounds__(1 << (L - 5), 1 << (15 - L)) srht_vec_kernel(const float* __restrict__ A, int64_t lda,
                                                                int64_t M, int64_t N,
                                                                const uint32_t* __restrict__ dbits,
                                                                const int* __restrict__ cols, int s,
                                                                float* __restrict__ C, int64_t ldc) {
    constexpr int T = 1 << (L - 5);
    constexpr int NP = 1 << L;
    extern __shared__ float4 smem4[];
    float* buf = reinterpret_cast<float*>(smem4);          // NP floats, swizzled
    int* scol = reinterpret_cast<int*>(buf + NP);
    for (int k = threadIdx.x; k < s; k += T) scol[k] = cols[k];
    const int j = threadIdx.x;
    const int64_t nwords = (N + 31) / 32;
    int o2[8], o3[8];
    sw_offsets(j, o2, o3);
    __syncthreads();

    for (int64_t row = blockIdx.x; row < M; row += gridDim.x) {
        const float* Ar = A + row * lda;
        float x[32];
        // phase 1: register e = 4 r + q  <->  logical bits (q: 0, 1; r: L-3 .. L-1)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int idx = r * 4 * T + 4 * j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx + 3 < N) {
                v = __ldg(reinterpret_cast<const float4*>(Ar + idx));
            } else if (idx < N) {
                v.x = __ldg(Ar + idx);
                if (idx + 1 < N) v.y = __ldg(Ar + idx + 1);
                if (idx + 2 < N) v.z = __ldg(Ar + idx + 2);
            }
            const uint32_t w = (idx >> 5) < nwords ? __ldg(dbits + (idx >> 5)) >> (idx & 31) : 0u;
            x[4 * r + 0] = __uint_as_float(__float_as_uint(v.x) ^ ((w & 1u) << 31));
            x[4 * r + 1] = __uint_as_float(__float_as_uint(v.y) ^ (((w >> 1) & 1u) << 31));
            x[4 * r + 2] = __uint_as_float(__float_as_uint(v.z) ^ (((w >> 2) & 1u) << 31));
            x[4 * r + 3] = __uint_as_float(__float_as_uint(v.w) ^ (((w >> 3) & 1u) << 31));
        }
        fwht32<5>(x);
#pragma unroll
        for (int r = 0; r < 8; ++r)
            *reinterpret_cast<float4*>(buf + phys_sw(r * 4 * T + 4 * j)) =
                make_float4(x[4 * r], x[4 * r + 1], x[4 * r + 2], x[4 * r + 3]);
        __syncthreads();
        // phase 2: register c <-> logical bits 2..6
        {
#pragma unroll
            for (int c = 0; c < 32; ++c) x[c] = buf[o2[c & 7] + 4 * (c & 24)];
            fwht32<5>(x);
#pragma unroll
            for (int c = 0; c < 32; ++c) buf[o2[c & 7] + 4 * (c & 24)] = x[c];
        }
        __syncthreads();
        // phase 3: register k <-> logical bits 7..11, butterflies on bits 7 .. L-4
        {
#pragma unroll
            for (int k = 0; k < 32; ++k) x[k] = buf[o3[k & 7] + 128 * k];
            fwht32<L - 10>(x);
#pragma unroll
            for (int k = 0; k < 32; ++k) buf[o3[k & 7] + 128 * k] = x[k];
        }
        __syncthreads();
        for (int k = j; k < s; k += T) C[row * ldc + k] = buf[phys_sw(scol[k])];
        __syncthreads();
    }
}

// HRTT outputs of one row held in buf (phys_sw layout, NP = 32 T coordinates)
// for s a power of two; htab holds the swizzled offset phys_sw(c) of each
// table entry with the sign in bit 15.  Thread j adds the 32 entries
// q = u T + j in the order of u.  For s >= T these land in its own buckets (u mod s/T) T + j, in
// bucket order; for s < T all in bucket j mod s, whose T/s partial sums (T/32
// after a shuffle reduction when s < 32) are then added through red.
template <int T>
__device__ __forceinline__ void hashed_outputs_pow2(const float* buf, const uint16_t* htab, int s, int j,
                                                    float* red, float* __restrict__ out) {
    auto term = [&](int u) {
        const uint32_t e = htab[u * T + j];
        const float v = buf[e & 0x7fffu];
        return __uint_as_float(__float_as_uint(v) ^ ((e << 16) & 0x80000000u));
    };
    if (s >= T) {                                        // uniform across the CTA: no barrier below
        const int V = s / T;
        for (int v = 0; v < V; ++v) {
            float acc = 0.0f;
            for (int u = v; u < 32; u += V) acc += term(u);
            out[v * T + j] = acc;
        }
        return;
    }
    float acc = 0.0f;
#pragma unroll
    for (int u = 0; u < 32; ++u) acc += term(u);
    if (s < 32) {
        // lanes with equal lane mod s share a bucket: fold the higher lane bits
        for (int off = 16; off >= s; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((j & 31) < s) red[(j >> 5) * s + (j & 31)] = acc;
    } else {
        red[j] = acc;
    }
    __syncthreads();
    if (j < s) {
        const int cnt = T / (s < 32 ? 32 : s);
        float t = 0.0f;
        for (int i = 0; i < cnt; ++i) t += red[i * s + j];
        out[j] = t;
    }
}

// Orders the table for hashed_outputs_pow2 (in place).  Thread j of the bulk
// kernel reads the entries at q = u T + j in the order of u; any order of a
// thread's entries that keeps u mod V (V = max(1, s/T)) keeps every entry in
// its bucket.  Step by step, the lanes of a warp take, lowest lane first, an
// unused entry whose shared-memory bank (of its swizzled offset) no lower lane
// took at this step; a lane left without such an entry takes its first unused
// one.  Deterministic; one warp per 32 threads of the bulk kernel's CTA.
template <int L>
__global__ void __launch_bounds__(32) hrtt_order_kernel(uint16_t* __restrict__ tbl, int s) {
    constexpr int T = 1 << (L - 5);
    const int lane = threadIdx.x;
    const int j = blockIdx.x * 32 + lane;
    const int V = s >= T ? s / T : 1;                 // 1 .. 32, a power of two
    uint32_t e[32], bank[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) {
        e[u] = tbl[u * T + j];
        bank[u] = (uint32_t)phys_sw((int)(e[u] & 0x7fffu)) & 31u;
    }
    uint32_t cls0 = 0;                                // entries u = 0 mod V
    for (int u = 0; u < 32; u += V) cls0 |= 1u << u;
    uint32_t rem = 0xffffffffu;
    for (int uo = 0; uo < 32; ++uo) {
        const uint32_t cls = cls0 << (uo % V);
        uint32_t taken = 0;
        int pick = -1;
        for (int round = 0; round < 32; ++round) {
            int cand = -1;
            if (pick < 0) {
                const uint32_t avail = rem & cls;
#pragma unroll
                for (int i = 31; i >= 0; --i)
                    if (((avail >> i) & 1u) && !((taken >> bank[i]) & 1u)) cand = i;
            }
            if (!__any_sync(0xffffffffu, cand >= 0)) break;
            uint32_t b = 32u + (uint32_t)lane;            // distinct for lanes without a candidate
#pragma unroll
            for (int i = 0; i < 32; ++i)
                if (i == cand) b = bank[i];
            const uint32_t grp = __match_any_sync(0xffffffffu, b);
            const bool win = cand >= 0 && (__ffs(grp) - 1) == lane;
            if (win) pick = cand;
            taken |= __reduce_or_sync(0xffffffffu, win ? (1u << b) : 0u);
        }
        if (pick < 0) pick = __ffs(rem & cls) - 1;        // every bank left is taken: accept a conflict
        uint32_t v = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (i == pick) v = e[i];
        tbl[uo * T + j] = (uint16_t)v;
        rem &= ~(1u << pick);
    }
}

// Bulk-copy form of srht_vec_kernel for rows of a multiple of 4 floats: each
// row arrives in shared memory by one bulk copy (cp.async.bulk, completion on an
// mbarrier) issued as soon as the previous row's gather is done; phase 1 then
// reads the row from shared memory (conflict-free 16-byte loads), and the same
// buffer serves the two transposes.  With one row buffer per CTA, 2^(15-L) CTAs
// share an SM, so one CTA's copy and barriers overlap the others' transforms.
// Waits are bounded in time; on expiry *err is set and the CTA drains its copy
// and returns.  HASH selects the HRTT outputs (table htab of NP entries, s a
// power of two) instead of the s sampled coordinates cols.
template <int L, bool HASH>
__global__ void __launch_bounds__(1 << (L - 5), 1 << (15 - L)) srht_bulk_kernel(
    const float* __restrict__ A, int64_t lda, int64_t M, int64_t N, const uint32_t* __restrict__ dbits,
    const int* __restrict__ cols, const uint16_t* __restrict__ htab_g, int s, float* __restrict__ C,
    int64_t ldc, int* err) {
    constexpr int T = 1 << (L - 5);
    constexpr int NP = 1 << L;
    extern __shared__ __align__(128) float4 smem4[];
    float* buf = reinterpret_cast<float*>(smem4);           // NP floats, swizzled
    int* scol = reinterpret_cast<int*>(buf + NP);           // s sampled coordinates (SRHT)
    uint16_t* htab = reinterpret_cast<uint16_t*>(buf + NP); // NP table entries (HRTT)
    float* red = buf + NP + NP / 2;                         // T partial sums (HRTT)
    __shared__ __align__(8) uint64_t full;
    const int j = threadIdx.x;
    const uint32_t row_bytes = (uint32_t)(N * 4);
    const int64_t nwords = (N + 31) / 32;
    int o2[8], o3[8];
    sw_offsets(j, o2, o3);
    if (j == 0) {
        tc::mbar_init(&full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (HASH) {
        for (int q = j; q < NP; q += T) {
            const uint32_t e = htab_g[q];
            htab[q] = (uint16_t)(phys_sw((int)(e & 0x7fffu)) | (e & 0x8000u));
        }
    } else {
        for (int k = j; k < s; k += T) scol[k] = cols[k];
    }
    __syncthreads();
    auto issue = [&](int64_t r) {
        tc::fence_proxy_async();                             // earlier generic accesses of buf first
        tc::mbar_arrive_expect_tx(&full, row_bytes);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                tc::smem_u32(buf)),
            "l"(A + r * lda), "r"(row_bytes), "r"(tc::smem_u32(&full))
            : "memory");
    };
    if (j == 0 && blockIdx.x < M) issue(blockIdx.x);
    int it = 0;
    for (int64_t row = blockIdx.x; row < M; row += gridDim.x, ++it) {
        // wait for this row's copy: the it-th completion of full
        bool ok = true;
        {
            const uint32_t par = (uint32_t)(it & 1);
            if (!tc::mbar_test(&full, par)) {
                const unsigned long long t0 = tc::now_ns();
                while (!tc::mbar_test_sleep(&full, par)) {
                    if (tc::now_ns() - t0 > tc::kWaitNs) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (j == 0) {
                if (err) atomicExch(err, 1);
                tc::mbar_drain(&full, (uint32_t)(it & 1));   // the one copy in flight
            }
            return;
        }
        float x[32];
        // phase 1: register e = 4 r + q  <->  logical bits (q: 0, 1; r: L-3 .. L-1)
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int idx = r * 4 * T + 4 * j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (idx < N) v = *reinterpret_cast<const float4*>(buf + idx);
            const uint32_t w = (idx >> 5) < nwords ? __ldg(dbits + (idx >> 5)) >> (idx & 31) : 0u;
            x[4 * r + 0] = __uint_as_float(__float_as_uint(v.x) ^ ((w & 1u) << 31));
            x[4 * r + 1] = __uint_as_float(__float_as_uint(v.y) ^ (((w >> 1) & 1u) << 31));
            x[4 * r + 2] = __uint_as_float(__float_as_uint(v.z) ^ (((w >> 2) & 1u) << 31));
            x[4 * r + 3] = __uint_as_float(__float_as_uint(v.w) ^ (((w >> 3) & 1u) << 31));
        }
        fwht32<5>(x);
        __syncthreads();                                      // every phase-1 read of buf is done
#pragma unroll
        for (int r = 0; r < 8; ++r)
            *reinterpret_cast<float4*>(buf + phys_sw(r * 4 * T + 4 * j)) =
                make_float4(x[4 * r], x[4 * r + 1], x[4 * r + 2], x[4 * r + 3]);
        __syncthreads();
        {
#pragma unroll
            for (int c = 0; c < 32; ++c) x[c] = buf[o2[c & 7] + 4 * (c & 24)];
            fwht32<5>(x);
#pragma unroll
            for (int c = 0; c < 32; ++c) buf[o2[c & 7] + 4 * (c & 24)] = x[c];
        }
        __syncthreads();
        {
#pragma unroll
            for (int k = 0; k < 32; ++k) x[k] = buf[o3[k & 7] + 128 * k];
            fwht32<L - 10>(x);
#pragma unroll
            for (int k = 0; k < 32; ++k) buf[o3[k & 7] + 128 * k] = x[k];
        }
        __syncthreads();
        if constexpr (HASH)
            hashed_outputs_pow2<T>(buf, htab, s, j, red, C + row * ldc);
        else
            for (int k = j; k < s; k += T) C[row * ldc + k] = buf[phys_sw(scol[k])];
        __syncthreads();                                      // every gather read of buf is done
        if (j == 0 && row + gridDim.x < M) issue(row + gridDim.x);
    }
}

template <int L, bool HASH>
cudaError_t launch_bulk(const MatView& A, const uint32_t* dbits, const int* cols, uint16_t* htab, int s,
                        float* C, int64_t ldc, int* err, cudaStream_t st);

template <int L>
cudaError_t launch_vec(const MatView& A, const uint32_t* dbits, const int* cols, int s, float* C,
                       int64_t ldc, cudaStream_t st);

int g_sm_count = 0;

int sm_count() {
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (!g_sm_count) g_sm_count = 148;
    }
    return g_sm_count;
}

template <int L>
cudaError_t launch_vec(const MatView& A, const uint32_t* dbits, const int* cols, int s, float* C,
                       int64_t ldc, cudaStream_t st) {
    constexpr int T = 1 << (L - 5);
    const size_t smem = sizeof(float) * ((size_t)1 << L) + sizeof(int) * (size_t)s;
    auto k = srht_vec_kernel<L>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(A.rows, (int64_t)std::max(per_sm, 1) * sm_count()));
    k<<<(unsigned)grid, T, smem, st>>>(static_cast<const float*>(A.ptr), A.ld, A.rows, A.cols, dbits, cols, s,
                                       C, ldc);
    return cudaGetLastError();
}

template <int L, bool HASH>
cudaError_t launch_bulk(const MatView& A, const uint32_t* dbits, const int* cols, uint16_t* htab, int s,
                        float* C, int64_t ldc, int* err, cudaStream_t st) {
    constexpr int T = 1 << (L - 5);
    if constexpr (HASH) {
        hrtt_order_kernel<L><<<T / 32, 32, 0, st>>>(htab, s);
        cudaError_t e0 = cudaGetLastError();
        if (e0 != cudaSuccess) return e0;
    }
    const size_t smem = sizeof(float) * ((size_t)1 << L) +
                        (HASH ? sizeof(uint16_t) * ((size_t)1 << L) + sizeof(float) * T : sizeof(int) * (size_t)s);
    auto k = srht_bulk_kernel<L, HASH>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(A.rows, (int64_t)std::max(per_sm, 1) * sm_count()));
    k<<<(unsigned)grid, T, smem, st>>>(static_cast<const float*>(A.ptr), A.ld, A.rows, A.cols, dbits, cols, htab,
                                       s, C, ldc, err);
    return cudaGetLastError();
}

template <int LOGN, bool TRANS, typename TA>
cudaError_t launch_reg(const MatView& A, const uint32_t* dbits, const int* cols, const uint16_t* htab, int hnp,
                       int s, float* C, int64_t ldc, cudaStream_t st) {
    constexpr int NP = 1 << LOGN;
    constexpr int T = 1 << (LOGN / 2);
    constexpr int G = 128 / T;
    constexpr int PITCH = NP + (T < 32 ? 16 : 0);
    const size_t smem = sizeof(float) * (size_t)G * PITCH + sizeof(uint32_t) * (NP / 32) +
                        sizeof(int) * (size_t)s;
    auto k = srht_reg_kernel<LOGN, TRANS, TA>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 128, smem);
    if (e != cudaSuccess) return e;
    const int64_t groups = (A.rows + G - 1) / G;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)std::max(per_sm, 1) * sm_count()));
    k<<<(unsigned)grid, 128, smem, st>>>(static_cast<const TA*>(A.ptr), A.ld, A.rows, A.cols, dbits,
                                         cols, htab, hnp, s, C, ldc);
    return cudaGetLastError();
}

// SRHT (cols, htab null) or HRTT (htab, cols null).
template <bool TRANS, typename TA>
cudaError_t launch_srht_t(const MatView& A, const uint32_t* dbits, const int* cols, uint16_t* htab, int s,
                          float* C, int64_t ldc, int* err, cudaStream_t st) {
    const int need = pow2_bits(A.cols);
    const int hnp = 1 << need;
    if constexpr (!TRANS && sizeof(TA) == 4) {
        if (err && need >= 12 && need <= 14 && (A.ld % 4) == 0 && (A.cols % 4) == 0 &&
            (reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0) {
            if (!htab) {
                if (need == 12) return launch_bulk<12, false>(A, dbits, cols, nullptr, s, C, ldc, err, st);
                if (need == 13) return launch_bulk<13, false>(A, dbits, cols, nullptr, s, C, ldc, err, st);
                return launch_bulk<14, false>(A, dbits, cols, nullptr, s, C, ldc, err, st);
            }
            if ((s & (s - 1)) == 0) {
                if (need == 12) return launch_bulk<12, true>(A, dbits, nullptr, htab, s, C, ldc, err, st);
                if (need == 13) return launch_bulk<13, true>(A, dbits, nullptr, htab, s, C, ldc, err, st);
                return launch_bulk<14, true>(A, dbits, nullptr, htab, s, C, ldc, err, st);
            }
        }
        if (!htab && need >= 12 && need <= 14 && (A.ld % 4) == 0 && (reinterpret_cast<uintptr_t>(A.ptr) & 15) == 0) {
            if (need == 12) return launch_vec<12>(A, dbits, cols, s, C, ldc, st);
            if (need == 13) return launch_vec<13>(A, dbits, cols, s, C, ldc, st);
            return launch_vec<14>(A, dbits, cols, s, C, ldc, st);
        }
    }
    if (need <= 8) return launch_reg<8, TRANS, TA>(A, dbits, cols, htab, hnp, s, C, ldc, st);
    if (need <= 10) return launch_reg<10, TRANS, TA>(A, dbits, cols, htab, hnp, s, C, ldc, st);
    if (need <= 12) return launch_reg<12, TRANS, TA>(A, dbits, cols, htab, hnp, s, C, ldc, st);
    if (need <= 14) return launch_reg<14, TRANS, TA>(A, dbits, cols, htab, hnp, s, C, ldc, st);
    if (need > 15) return cudaErrorNotSupported;
    const size_t smem = sizeof(float) << need;
    auto k = srht_smem_kernel<TRANS, TA>;
    cudaError_t e = allow_dynamic_smem(reinterpret_cast<const void*>(k));
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(A.rows, (int64_t)sm_count() * 1);
    k<<<(unsigned)grid, 1024, smem, st>>>(static_cast<const TA*>(A.ptr), A.ld, A.rows, A.cols, need,
                                          dbits, cols, htab, s, C, ldc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_right_srht(const MatView& A, const uint32_t* dbits, const int* cols, int s,
                              float* C, int64_t ldc, cudaStream_t st, int* err) {
    if (s <= 0 || A.rows <= 0) return cudaSuccess;
    if (A.dtype == RE_F32)
        return A.trans ? launch_srht_t<true, float>(A, dbits, cols, nullptr, s, C, ldc, err, st)
                       : launch_srht_t<false, float>(A, dbits, cols, nullptr, s, C, ldc, err, st);
    return A.trans ? launch_srht_t<true, double>(A, dbits, cols, nullptr, s, C, ldc, err, st)
                   : launch_srht_t<false, double>(A, dbits, cols, nullptr, s, C, ldc, err, st);
}

cudaError_t launch_right_hrtt(const MatView& A, const uint32_t* dbits, uint16_t* tbl, int s,
                              float* C, int64_t ldc, cudaStream_t st, int* err) {
    if (s <= 0 || A.rows <= 0) return cudaSuccess;
    if (!tbl || s > (int64_t(1) << pow2_bits(A.cols))) return cudaErrorInvalidValue;
    if (A.dtype == RE_F32)
        return A.trans ? launch_srht_t<true, float>(A, dbits, nullptr, tbl, s, C, ldc, err, st)
                       : launch_srht_t<false, float>(A, dbits, nullptr, tbl, s, C, ldc, err, st);
    return A.trans ? launch_srht_t<true, double>(A, dbits, nullptr, tbl, s, C, ldc, err, st)
                   : launch_srht_t<false, double>(A, dbits, nullptr, tbl, s, C, ldc, err, st);
}

}  // namespace re
