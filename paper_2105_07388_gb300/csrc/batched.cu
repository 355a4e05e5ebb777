// Batched Algorithm 1 (Sec. 5) over many independent blocks, e.g. the
// off-diagonal blocks of a hierarchical matrix (Sec. 1 motivates rank
// estimation for low-rank off-diagonal blocks).
//
// Level-synchronous: every still-active block advances together through the
// sketch-width ladder s = s0, 2 s0, ..., one level at a time, and each level is
// a fixed sequence of batched kernels over all blocks:
//   generator     X_b columns [s_prev, s) for every active block (own seed each)
//   right sketch  one CTA per (block, row tile) work item (FP32 CUDA cores), or
//                 the persistent tcgen05 kernel (BF16x3); on the tensor-core
//                 path the first pass appends up to w1 columns at once, so the
//                 widths up to w1 cost one read of each block
//   left sketch   one CTA per (block, core tile sized to the request), Y_b
//                 generated on the fly
//   core sigma    one CTA per block (QR + one-sided Jacobi in shared memory)
//   read-off      one thread per block; converged blocks, and blocks that reached
//                 their largest width, retire by clearing their active flag
// Inactive blocks cost each kernel only a flag test.  The whole ladder is
// captured once into a CUDA graph and replayed for identical batches, so an
// estimate of thousands of uneven blocks is one graph launch with no host
// round trips.  Autotuners, run on the batch at hand and cached with its graph:
// on CUDA cores the right sketch's tile height (64 or 128 rows) per sketch width;
// on the tensor cores the first pass's width w1 (s0, 2 s0, ... up to the X^T
// pool), i.e. the N tile of the first pass -- a wider first pass costs little more
// than a narrow one (it is bound by reading the blocks) and spares later passes
// for the blocks that need them, but its tensor work grows; the ladders of every
// candidate give the same bits, so the fastest is kept.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace re {

namespace {

struct DBuf {
    void* p = nullptr;
    size_t cap = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= cap) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 256));
        if (e == cudaSuccess) cap = std::max<size_t>(bytes, 256);
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

__device__ __forceinline__ int find_prefix(const int64_t* prefix, int count, int64_t item) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void init_active_kernel(const int* valid, int* active, int* status, int count, int* tcerr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b == 0 && tcerr) *tcerr = 0;
    if (b >= count) return;
    active[b] = valid[b];
    status[b] = 0;
}

// X_b[k][j] (row-major, ld = s) for columns [col0, col0 + s) of every active block.
__global__ void gauss_x_batched_kernel(const BatchDesc* __restrict__ d, int count,
                                       const int64_t* __restrict__ col_prefix,
                                       const int* __restrict__ active, int col0, int s,
                                       float* __restrict__ Xpool) {
    const int ng = s / 4;
    const int64_t total = col_prefix[count] * ng;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t krow = idx / ng;
        const int b = find_prefix(col_prefix, count, krow);
        if (!active[b]) continue;
        const int64_t k = krow - col_prefix[b];
        const int g = (int)(idx % ng);
        float z[4];
        normals4((uint32_t)k, (uint32_t)(col0 / 4 + g), kStreamGX, d[b].seed, z);
        float* X = Xpool + d[b].x_off + k * s + 4 * g;
        *reinterpret_cast<float4*>(X) = make_float4(z[0], z[1], z[2], z[3]);
    }
}

// core_b[row0 + r][col0 + c] = sum_i Y_b[row0 + r][i] AX_b[i][col0 + c] over all
// rows i of block b; one CTA per (block, 64 x 64 tile), FP32 accumulation.
// Left sketch of the batched estimate (Algorithm 1 steps 4-6 per block), one CTA
// per (block, TR x TC core tile): core[row0 + r][col0 + c] = sum_i Y[row0 + r][i]
// AX[i][col0 + c] over the block's rows i.  The tile is sized to the request
// (TR = 16..64 rows, TC = 8..64 columns, 4 x 4 outputs per thread), and the 256
// threads split each chunk of rows into KS = 256 / (TR TC / 16) interleaved
// slices whose partial sums are added in a fixed order at the end.  A chunk
// generates TR x KC normals of Y (KC = 2048 / TR rows, the same work for every
// tile height) and reads KC x TC floats of AX.
template <int TR, int TC>
__global__ void __launch_bounds__(256, 3) left_batched_kernel(
    const BatchDesc* __restrict__ d, const int* __restrict__ active, const float* __restrict__ AXpool,
    int64_t ldax, double* __restrict__ corepool, int64_t core_stride, int ld_core, int row0, int R,
    int col0, int S, int tiles_c) {
    constexpr int KC = 2048 / TR;                  // rows of the block per chunk
    constexpr int OTX = TC / 4, OT = (TR / 4) * OTX;   // output threads
    constexpr int KS = 256 / OT;                   // row slices
    __shared__ __align__(16) float Ys[KC][TR + 4];
    __shared__ __align__(16) float Xs[KC][TC + 4];
    __shared__ __align__(16) float red[KS > 1 ? KS : 1][KS > 1 ? OT : 1][16];
    const int b = blockIdx.x;
    if (!active[b]) return;
    const BatchDesc D = d[b];
    const int rt = blockIdx.y / tiles_c, ct = blockIdx.y % tiles_c;
    const int tid = threadIdx.x;
    const int o = tid % OT, ks = tid / OT;
    const int ty = o / OTX, tx = o % OTX;
    const int qbase = row0 + rt * TR;             // a multiple of 4
    const float* AX = AXpool + D.ax_off;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    for (int64_t i0 = 0; i0 < D.rows; i0 += KC) {
        // Y tile: (TR / 4) x KC groups of four normals, two per thread
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tid + 256 * h;
            const int k = c % KC, g = c / KC;
            const int64_t i = i0 + k;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (i < D.rows && rt * TR + 4 * g < R)
                normals4((uint32_t)i, (uint32_t)((qbase >> 2) + g), kStreamGY, D.seed, z);
            *reinterpret_cast<float4*>(&Ys[k][4 * g]) = make_float4(z[0], z[1], z[2], z[3]);
        }
        // AX tile: KC x TC, consecutive threads along a row of AX
#pragma unroll
        for (int idx = tid; idx < KC * TC; idx += 256) {
            const int k = idx / TC, c = idx % TC;
            const int64_t i = i0 + k;
            const int cc = ct * TC + c;
            Xs[k][c] = (i < D.rows && cc < S) ? __ldg(AX + i * ldax + col0 + cc) : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = ks; k < KC; k += KS) {
            const float4 yv = *reinterpret_cast<const float4*>(&Ys[k][ty * 4]);
            const float4 xv = *reinterpret_cast<const float4*>(&Xs[k][tx * 4]);
            const float y[4] = {yv.x, yv.y, yv.z, yv.w};
            const float x[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fmaf(y[a], x[c], acc[a][c]);
        }
        __syncthreads();
    }
    double* core = corepool + (int64_t)b * core_stride;
    if constexpr (KS > 1) {
        // slice partial sums, added in slice order; one output per thread
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) red[ks][o][4 * a + c] = acc[a][c];
        __syncthreads();
        for (int idx = tid; idx < OT * 16; idx += 256) {
            const int oo = idx >> 4, a = (idx >> 2) & 3, c = idx & 3;
            float t = red[0][oo][idx & 15];
            for (int u = 1; u < KS; ++u) t += red[u][oo][idx & 15];
            const int r = rt * TR + (oo / OTX) * 4 + a;
            const int cc = ct * TC + (oo % OTX) * 4 + c;
            if (r < R && cc < S) core[(int64_t)(row0 + r) * ld_core + col0 + cc] = (double)t;
        }
    } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int r = rt * TR + ty * 4 + a;
            if (r >= R) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int cc = ct * TC + tx * 4 + c;
                if (cc < S) core[(int64_t)(row0 + r) * ld_core + col0 + cc] = (double)acc[a][c];
            }
        }
    }
}

template <int TR, int TC>
cudaError_t launch_left_batched_t(const BatchDesc* d, const int* active, int count, const float* AX, int64_t ldax,
                                  double* core, int64_t core_stride, int ld_core, int row0, int R, int col0, int S,
                                  cudaStream_t st) {
    const int tr = (R + TR - 1) / TR, tc = (S + TC - 1) / TC;
    left_batched_kernel<TR, TC><<<dim3(count, tr * tc), 256, 0, st>>>(d, active, AX, ldax, core, core_stride,
                                                                      ld_core, row0, R, col0, S, tc);
    return cudaGetLastError();
}

// TC <= TR (the ladder's requests have R >= 2 S; wider ones take more column tiles)
template <int TR>
cudaError_t launch_left_batched_r(const BatchDesc* d, const int* active, int count, const float* AX, int64_t ldax,
                                  double* core, int64_t core_stride, int ld_core, int row0, int R, int col0, int S,
                                  cudaStream_t st) {
    if (S >= 64 && TR >= 64) return launch_left_batched_t<TR, (TR >= 64 ? 64 : TR)>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
    if (S >= 32 && TR >= 32) return launch_left_batched_t<TR, (TR >= 32 ? 32 : TR)>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
    if (S >= 16 && TR >= 16) return launch_left_batched_t<TR, 16>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
    return launch_left_batched_t<TR, 8>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
}

// Core block rows [row0, row0 + R) x columns [col0, col0 + S) of every active block.
cudaError_t launch_left_batched(const BatchDesc* d, const int* active, int count, const float* AX, int64_t ldax,
                                double* core, int64_t core_stride, int ld_core, int row0, int R, int col0, int S,
                                cudaStream_t st) {
    if (R <= 0 || S <= 0 || count <= 0) return cudaSuccess;
    if (R >= 64) return launch_left_batched_r<64>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
    if (R >= 32) return launch_left_batched_r<32>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
    return launch_left_batched_r<16>(d, active, count, AX, ldax, core, core_stride, ld_core, row0, R, col0, S, st);
}

// Read-off for every active block at width s (Algorithm 1 step 8); retires blocks.
__global__ void readoff_batched_kernel(const BatchDesc* __restrict__ d, int count, int* active,
                                       const double* __restrict__ sigma, int64_t sstride, int s, int r1,
                                       double scale, double eps, double norm_a, int* status,
                                       DevReadoff* out, double* sigma_scaled, int* final_s, const int* tcerr) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count || !active[b]) return;
    const double* sg = sigma + (int64_t)b * sstride;
    double* ss = sigma_scaled + (int64_t)b * sstride;
    DevReadoff r;
    // a bounded wait of the tensor-core sketch expired: every block reports it
    r.status = (tcerr && *tcerr) ? RE_ERR_TIMEOUT : status[b];
    r.sweeps = 0;
    for (int i = 0; i < r1; ++i) ss[i] = sg[i] * scale;
    const double ref = norm_a > 0.0 ? norm_a : ss[0];
    r.tau = eps * ref;
    r.rank = -1;
    for (int i = 0; i < r1; ++i)
        if (ss[i] <= r.tau) {
            r.rank = i;
            break;
        }
    int gi = 1;
    double gr = r1 >= 2 ? -1.0 : 1.0;
    for (int i = 1; i < r1; ++i) {
        const double a = ss[i - 1], c = ss[i];
        const double ratio = c > 0.0 ? a / c : (a > 0.0 ? INFINITY : 1.0);
        if (ratio > gr) {
            gr = ratio;
            gi = i;
        }
    }
    r.gap_index = gi;
    r.gap_ratio = gr;
    out[b] = r;
    final_s[b] = s;
    if (r.status != RE_OK || r.rank >= 0 || 2 * s > d[b].smax || r1 >= d[b].cols) active[b] = 0;
}

int r1_of(int s) {
    int r = 1;
    while ((2 * 11 * (r + 1) + 10) / 20 <= s) ++r;
    return r;
}

}  // namespace

struct BatchedState {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, t0 = nullptr, t1 = nullptr;
    DBuf ax, x, xt, tcerr, actpre, core, sigma, sscaled, status, out, active, valid, descs, pre128, pre64, colpre, finals;
    DBuf tmaps;                       // tensor-core path: four row-class tensor maps per block
    DBuf tileblk;                     // tensor-core path: block of each active 128-row tile
    cudaGraphExec_t exec = nullptr;
    std::vector<unsigned char> key;
    int bm_for[16] = {0};
    int w1 = 0;                       // tensor-core path: width of the ladder's first pass
    int64_t launches_per_run = 0;
};

void batched_destroy(BatchedState* st) {
    if (!st) return;
    if (st->exec) cudaGraphExecDestroy(st->exec);
    DBuf* bufs[] = {&st->ax, &st->x, &st->xt, &st->tcerr, &st->actpre, &st->core, &st->sigma, &st->sscaled, &st->status, &st->out,
                    &st->active, &st->valid, &st->descs, &st->pre128, &st->pre64, &st->colpre, &st->finals, &st->tmaps,
                    &st->tileblk};
    for (DBuf* b : bufs) b->release();
    if (st->ev_in) cudaEventDestroy(st->ev_in);
    if (st->ev_out) cudaEventDestroy(st->ev_out);
    if (st->t0) cudaEventDestroy(st->t0);
    if (st->t1) cudaEventDestroy(st->t1);
    if (st->stream) cudaStreamDestroy(st->stream);
    delete st;
}

int batched_estimate(BatchedState** pst, const re_opts& o, const re_block* blocks, const re_kblock* kblocks,
                     int count, double eps, uint64_t seed, double* sigma_out, int sigma_cap, re_result* out,
                     cudaStream_t ustream, int64_t* launches) {
    if (!*pst) {
        BatchedState* st = new BatchedState();
        if (cudaStreamCreateWithFlags(&st->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&st->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&st->ev_out, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&st->t0) != cudaSuccess || cudaEventCreate(&st->t1) != cudaSuccess) {
            batched_destroy(st);
            return set_last_error(RE_ERR_CUDA, "batched: stream/event creation failed");
        }
        *pst = st;
    }
    BatchedState* st = *pst;
    const int s0 = o.s0;
    const int scap = std::min(o.s_max, 128);
    // ---- host descriptors
    std::vector<BatchDesc> hd(count);
    std::vector<int> valid(count, 0), transposed(count, 0);
    std::vector<int64_t> pre128(count + 1, 0), pre64(count + 1, 0), colpre(count + 1, 0);
    int S_MAX = 0;
    for (int i = 0; i < count; ++i) {
        BatchDesc& D = hd[i];
        std::memset(&D, 0, sizeof(D));
        int64_t m = 0, n = 0;
        bool ok;
        if (kblocks) {
            // matrix-free: orient by swapping the point sets (the kernel is symmetric)
            const re_kblock& B = kblocks[i];
            m = B.m;
            n = B.n;
            ok = B.x && B.y && m > 0 && n > 0 && m <= INT32_MAX && n <= INT32_MAX;
            if (ok) {
                D.px = m >= n ? B.x : B.y;
                D.py = m >= n ? B.y : B.x;
            }
        } else {
            const re_block& B = blocks[i];
            m = B.m;
            n = B.n;
            ok = B.ptr && m > 0 && n > 0 && B.ld >= n && m <= INT32_MAX && n <= INT32_MAX;
            if (ok) {
                D.A = static_cast<const float*>(B.ptr);
                D.ld = B.ld;
                D.trans = m < n;
            }
        }
        if (ok) {
            transposed[i] = m < n;
            D.rows = std::max(m, n);
            D.cols = std::min(m, n);
            int sm = s0;
            while (sm * 2 <= scap) sm *= 2;
            D.smax = sm;
            S_MAX = std::max(S_MAX, sm);
            valid[i] = 1;
        }
        D.seed = seed + (uint64_t)i;
    }
    if (S_MAX == 0) S_MAX = s0;
    const int SNEW = std::max(s0, S_MAX / 2);
    // BF16x3 split products on the tensor cores (X^T pool of tc_mma_n rows per block),
    // otherwise FP32 CUDA cores with an autotuned tile height
    const bool use_tc = o.precision == RE_PREC_BF16X3;
    const int NXT = tc_mma_n(SNEW);
    // row-major stored blocks on the tensor-core path: four row-class tensor maps each
    const size_t mapb = row_class_map_bytes();
    std::vector<unsigned char> hmaps;
    if (use_tc && !kblocks) {
        hmaps.assign((size_t)count * 4 * mapb, 0);
        for (int i = 0; i < count; ++i) {
            BatchDesc& D = hd[i];
            // row-major: 36 floats (32 values and up to 3 before) x 32 rows per class and
            // half chunk; stored transposed: 132 floats (128 oriented rows and up to 3
            // before) x 8 stored rows
            if (valid[i] && D.A && !D.trans)
                D.tmaps = encode_row_class_maps(D.A, D.ld, D.rows, D.cols, 36, 32,
                                                hmaps.data() + (size_t)i * 4 * mapb) ? 1 : 0;
            else if (valid[i] && D.A && D.trans)
                D.tmaps = encode_row_class_maps(D.A, D.ld, D.cols, D.rows, 132, 8,
                                                hmaps.data() + (size_t)i * 4 * mapb) ? 2 : 0;
        }
    }
    int64_t ax_total = 0, x_total = 0, xt_total = 0;
    for (int i = 0; i < count; ++i) {
        BatchDesc& D = hd[i];
        D.ax_off = ax_total;
        D.x_off = x_total;
        D.kpad = (D.cols + 63) / 64 * 64;
        D.xt_off = xt_total;
        ax_total += D.rows * S_MAX;
        x_total += (D.cols * SNEW + 63) / 64 * 64;
        if (use_tc && valid[i]) xt_total += (int64_t)NXT * D.kpad;
        pre128[i + 1] = pre128[i] + (valid[i] ? (D.rows + 127) / 128 : 0);
        pre64[i + 1] = pre64[i] + (valid[i] ? (D.rows + 63) / 64 : 0);
        colpre[i + 1] = colpre[i] + (valid[i] ? D.cols : 0);
    }
    const int64_t core_stride = 2LL * S_MAX * S_MAX;
    cudaError_t e = cudaSuccess;
    auto ens = [&](DBuf& b, size_t bytes) {
        if (e == cudaSuccess) e = b.ensure(bytes);
    };
    ens(st->ax, sizeof(float) * (size_t)std::max<int64_t>(ax_total, 1));
    if (use_tc) {
        ens(st->xt, sizeof(uint16_t) * (size_t)std::max<int64_t>(xt_total, 1));
        ens(st->tcerr, sizeof(int));
        ens(st->actpre, sizeof(int64_t) * (size_t)(count + 1));
        ens(st->tileblk, sizeof(int) * (size_t)std::max<int64_t>(pre128[count], 1));
    } else {
        ens(st->x, sizeof(float) * (size_t)std::max<int64_t>(x_total, 1));
    }
    ens(st->core, sizeof(double) * (size_t)core_stride * count);
    ens(st->sigma, sizeof(double) * (size_t)S_MAX * count);
    ens(st->sscaled, sizeof(double) * (size_t)S_MAX * count);
    ens(st->status, sizeof(int) * (size_t)count);
    ens(st->out, sizeof(DevReadoff) * (size_t)count);
    ens(st->active, sizeof(int) * (size_t)count);
    ens(st->valid, sizeof(int) * (size_t)count);
    ens(st->descs, sizeof(BatchDesc) * (size_t)count);
    ens(st->pre128, sizeof(int64_t) * (size_t)(count + 1));
    ens(st->pre64, sizeof(int64_t) * (size_t)(count + 1));
    ens(st->colpre, sizeof(int64_t) * (size_t)(count + 1));
    ens(st->finals, sizeof(int) * (size_t)count);
    if (!hmaps.empty()) ens(st->tmaps, hmaps.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_last_error(RE_ERR_NOMEM, "batched: device workspace allocation failed");
    }
    // cache key: everything the captured graph depends on
    std::vector<unsigned char> key;
    auto put = [&](const void* p, size_t n) {
        const unsigned char* c = static_cast<const unsigned char*>(p);
        key.insert(key.end(), c, c + n);
    };
    put(&count, sizeof(count));
    put(&eps, sizeof(eps));
    put(&o, sizeof(o));
    put(hd.data(), sizeof(BatchDesc) * hd.size());
    put(valid.data(), sizeof(int) * valid.size());
    const void* pools[] = {st->ax.p, st->x.p, st->xt.p, st->tcerr.p, st->actpre.p, st->core.p, st->sigma.p, st->sscaled.p,
                           st->status.p, st->out.p, st->active.p, st->finals.p, st->tmaps.p, st->tileblk.p};
    put(pools, sizeof(pools));

    cudaStream_t bs = st->stream;
    BatchDesc* dd = st->descs.as<BatchDesc>();
    int* active = st->active.as<int>();
    int* status = st->status.as<int>();
    if (!st->exec || key != st->key) {
        if (st->exec) {
            cudaGraphExecDestroy(st->exec);
            st->exec = nullptr;
        }
        e = cudaMemcpy(dd, hd.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(st->valid.p, valid.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(st->pre128.p, pre128.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(st->pre64.p, pre64.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(st->colpre.p, colpre.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !hmaps.empty()) e = cudaMemcpy(st->tmaps.p, hmaps.data(), hmaps.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, "batched: descriptor upload failed");
        // ---- autotune the right-sketch tile height for each width of the ladder
        // (CUDA-core path; the candidates differ only in tiling, not in arithmetic)
        if (!use_tc) {
            init_active_kernel<<<(count + 255) / 256, 256, 0, bs>>>(st->valid.as<int>(), active, status, count,
                                                                    nullptr);
            for (int s_prev = 0, s = s0; s <= S_MAX; s_prev = s, s *= 2) {
                const int sn = s - s_prev;
                const int slot = 31 - __builtin_clz((unsigned)sn);
                if (st->bm_for[slot]) continue;
                gauss_x_batched_kernel<<<1024, 256, 0, bs>>>(dd, count, st->colpre.as<int64_t>(), active, s_prev, sn,
                                                            st->x.as<float>());
                float best = 1e30f;
                int best_bm = 128;
                for (int bm : {128, 64}) {
                    const int64_t* pre = bm == 128 ? st->pre128.as<int64_t>() : st->pre64.as<int64_t>();
                    const int64_t items = bm == 128 ? pre128[count] : pre64[count];
                    for (int rep = 0; rep < 2; ++rep) {     // first run warms up
                        cudaEventRecord(st->t0, bs);
                        e = launch_right_simt_batched(dd, count, pre, items, active, st->x.as<float>(), sn,
                                                      st->ax.as<float>(), S_MAX, s_prev, bm, bs);
                        cudaEventRecord(st->t1, bs);
                        if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, "batched: autotune launch failed");
                        cudaEventSynchronize(st->t1);
                    }
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, st->t0, st->t1);
                    if (ms < best) {
                        best = ms;
                        best_bm = bm;
                    }
                }
                st->bm_for[slot] = best_bm;
            }
            e = cudaStreamSynchronize(bs);
            if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, "batched: autotune failed");
        }
        // ---- capture the whole ladder.  Tensor-core path: the first pass appends the
        // right sketch up to w1 columns (within the X^T pool's SNEW rows) in one read
        // of every block; the later ladder widths up to w1 then need no pass over A.
        // Column j of AX does not depend on which pass computes it, so every width
        // sees the same AX whatever w1 is: the results are the same bits, only the
        // number of passes (and the time) changes.
        auto capture = [&](int w1, cudaGraphExec_t* exec, int64_t* nl_out) -> cudaError_t {
            cudaGraph_t graph = nullptr;
            cudaError_t ec = cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal);
            if (ec != cudaSuccess) return ec;
            int64_t nl = 0;
            int* tcerr = use_tc ? st->tcerr.as<int>() : nullptr;
            init_active_kernel<<<(count + 255) / 256, 256, 0, bs>>>(st->valid.as<int>(), active, status, count, tcerr);
            ++nl;
            int covered = 0;                          // AX columns computed so far
            cudaError_t el = cudaSuccess;
            for (int s_prev = 0, s = s0; s <= S_MAX && el == cudaSuccess; s_prev = s, s *= 2) {
                const int sn = s - s_prev;
                if (use_tc) {
                    if (s > covered) {
                        const int upto = covered == 0 ? std::max(s, w1) : s;
                        const int c0 = covered, cn = upto - covered;
                        el = launch_gauss_xt_batched(dd, count, active, c0, cn, tc_mma_n(cn), st->xt.as<uint16_t>(), bs);
                        if (el == cudaSuccess)
                            el = launch_compact_tiles(dd, count, active, st->actpre.as<int64_t>(),
                                                      st->tileblk.as<int>(), pre128[count], bs);
                        if (el == cudaSuccess)
                            el = launch_right_tc_batched(dd, count, st->actpre.as<int64_t>(), st->tileblk.as<int>(),
                                                         pre128[count],
                                                         st->xt.as<uint16_t>(), cn, st->ax.as<float>(), S_MAX, c0, tcerr,
                                                         st->tmaps.p, bs);
                        covered = upto;
                        nl += 4;
                    }
                } else {
                    const int bm = st->bm_for[31 - __builtin_clz((unsigned)sn)] == 64 ? 64 : 128;
                    gauss_x_batched_kernel<<<1024, 256, 0, bs>>>(dd, count, st->colpre.as<int64_t>(), active, s_prev, sn,
                                                                st->x.as<float>());
                    el = launch_right_simt_batched(dd, count, bm == 128 ? st->pre128.as<int64_t>() : st->pre64.as<int64_t>(),
                                                   bm == 128 ? pre128[count] : pre64[count], active, st->x.as<float>(), sn,
                                                   st->ax.as<float>(), S_MAX, s_prev, bm, bs);
                    nl += 2;
                }
                if (el != cudaSuccess) break;
                if (s_prev > 0) {
                    el = launch_left_batched(dd, active, count, st->ax.as<float>(), S_MAX, st->core.as<double>(),
                                             core_stride, S_MAX, 2 * s_prev, 2 * sn, 0, s_prev, bs);
                    ++nl;
                    if (el != cudaSuccess) break;
                }
                el = launch_left_batched(dd, active, count, st->ax.as<float>(), S_MAX, st->core.as<double>(),
                                         core_stride, S_MAX, 0, 2 * s, s_prev, sn, bs);
                ++nl;
                if (el != cudaSuccess) break;
                el = launch_core_sigma_batched(st->core.as<double>(), 2 * s, s, S_MAX, core_stride, count,
                                               st->sigma.as<double>(), S_MAX, status, bs, active);
                ++nl;
                if (el != cudaSuccess) break;
                readoff_batched_kernel<<<(count + 127) / 128, 128, 0, bs>>>(
                    dd, count, active, st->sigma.as<double>(), S_MAX, s, std::min(r1_of(s), s),
                    1.0 / std::sqrt((double)s * (double)(2 * s)), eps, o.norm_a, status, st->out.as<DevReadoff>(),
                    st->sscaled.as<double>(), st->finals.as<int>(), tcerr);
                ++nl;
            }
            ec = cudaStreamEndCapture(bs, &graph);
            if (el == cudaSuccess) el = ec;
            if (el == cudaSuccess) el = cudaGraphInstantiate(exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            *nl_out = nl;
            return el;
        };
        // ---- autotune the first-pass width of the tensor-core ladder on this batch:
        // each candidate ladder is captured and timed once after a warm-up run (the
        // candidates give identical results, so the fastest is kept)
        std::vector<int> cands;
        if (use_tc) {
            if (o.batch_first_width > 0) {
                cands.push_back(std::min(std::max(o.batch_first_width, s0), std::min(SNEW, S_MAX)));
            } else {
                for (int w = s0; w <= SNEW && w <= S_MAX; w *= 2) cands.push_back(w);
            }
        } else {
            cands.push_back(s0);
        }
        float best = 1e30f;
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            cudaGraphExec_t ex = nullptr;
            int64_t nl = 0;
            e = capture(cands[ci], &ex, &nl);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (ex) cudaGraphExecDestroy(ex);
                if (st->exec) cudaGraphExecDestroy(st->exec);
                st->exec = nullptr;
                return set_last_error(RE_ERR_CUDA, "batched: graph capture failed");
            }
            float ms = 0.f;
            if (cands.size() > 1) {
                e = cudaGraphLaunch(ex, bs);
                if (e == cudaSuccess) e = cudaEventRecord(st->t0, bs);
                if (e == cudaSuccess) e = cudaGraphLaunch(ex, bs);
                if (e == cudaSuccess) e = cudaEventRecord(st->t1, bs);
                if (e == cudaSuccess) e = cudaEventSynchronize(st->t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, st->t0, st->t1);
                if (e != cudaSuccess) {
                    cudaGraphExecDestroy(ex);
                    return set_last_error(RE_ERR_CUDA, "batched: first-pass autotune failed");
                }
            }
            if (ms < best) {
                best = ms;
                if (st->exec) cudaGraphExecDestroy(st->exec);
                st->exec = ex;
                st->w1 = cands[ci];
                st->launches_per_run = nl;
            } else {
                cudaGraphExecDestroy(ex);
            }
        }
        st->key = key;
    }
    // ---- one graph launch, ordered after the caller's stream
    e = cudaEventRecord(st->ev_in, ustream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, st->ev_in, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(st->exec, bs);
    if (e == cudaSuccess) e = cudaEventRecord(st->ev_out, bs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ustream, st->ev_out, 0);
    if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, "batched: graph launch failed");
    *launches += st->launches_per_run;
    std::vector<DevReadoff> ro(count);
    std::vector<int> fin(count);
    e = cudaMemcpyAsync(ro.data(), st->out.p, sizeof(DevReadoff) * count, cudaMemcpyDeviceToHost, ustream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(fin.data(), st->finals.p, sizeof(int) * count, cudaMemcpyDeviceToHost, ustream);
    std::vector<double> sg;
    if (e == cudaSuccess && sigma_out && sigma_cap > 0) {
        sg.resize((size_t)count * S_MAX);
        e = cudaMemcpyAsync(sg.data(), st->sscaled.p, sizeof(double) * sg.size(), cudaMemcpyDeviceToHost, ustream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ustream);
    if (e != cudaSuccess) return set_last_error(RE_ERR_CUDA, "batched: result copy failed");
    for (int i = 0; i < count; ++i) {
        re_result& R = out[i];
        std::memset(&R, 0, sizeof(R));
        if (!valid[i]) {
            R.status = RE_ERR_ARG;
            continue;
        }
        const int s = fin[i];
        const int r1 = std::min(r1_of(s), s);
        const bool conv = ro[i].rank >= 0;
        R.status = ro[i].status == RE_OK ? RE_OK : ro[i].status;
        R.rank = conv ? ro[i].rank : r1;
        R.gap_index = ro[i].gap_index;
        R.gap_ratio = ro[i].gap_ratio;
        R.tau = ro[i].tau;
        R.n_sigma = r1;
        R.final_s = s;
        // passes over A: one per right-sketch pass the block took part in (on the
        // tensor-core path the first pass covers the widths up to w1)
        const int w1 = use_tc ? st->w1 : s0;
        int passes = 1;
        for (int t = 2 * w1; t <= s; t *= 2) ++passes;
        R.passes = passes;
        R.flags = (conv ? RE_CONVERGED : RE_LOWER_BOUND_ONLY) | (transposed[i] ? RE_TRANSPOSED : 0u);
        if (!sg.empty()) {
            const int nc = std::min(r1, sigma_cap);
            for (int j = 0; j < nc; ++j) sigma_out[(size_t)i * sigma_cap + j] = sg[(size_t)i * S_MAX + j];
        }
    }
    return RE_OK;
}

}  // namespace re
