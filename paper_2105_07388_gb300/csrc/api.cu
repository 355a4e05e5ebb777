// C ABI of librankest: handles, workspace, and the host side of Algorithm 1
// (Sec. 5): the adaptive loop that grows the sketch width by doubling and
// appending columns of X / rows of Y until the read-off of step 8 finds a
// trusted sketched singular value below eps*||A||.  Every numerical step runs
// in this library's kernels; the host only launches them and reads back a
// 40-byte read-off record per step.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>


#include "common.cuh"
#include "internal.h"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return RE_ERR_CUDA;
}

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

}  // namespace

enum Stage { kStageRight = 0, kStageLeft = 1, kStageSvd = 2, kStageOther = 3, kStageQbPre = 4, kStageQbOrth = 5,
             kStageQbProduct = 6 };

struct PendingTiming {
    int stage;
    cudaEvent_t a, b;
    double bytes, flops;
};

struct re_handle_ {
    int device = 0;
    re_opts opts{};
    bool timing = false;
    re_stats stats{};
    std::vector<PendingTiming> pending;
    std::vector<cudaEvent_t> event_pool;
    DevBuf x, xt, ax, part, core, sigma, sigma_scaled, svdws, acopy, dx, px, dy, py, ro, status, ht, fz;
    DevBuf qbws, qbsel;                 // Algorithm 3: factorization workspace, selection record
    DevBuf ctab;                        // cosine table of the SRCT left embedding
    DevBuf ctabx;                       // cosine table of the HRCT right embedding
    // precision mode (exact-product sketches): row exponents of A, digit slices of X
    // and Y, int64 accumulators of the right and left sketches, A X as FP32 pair planes
    // (transposed) with column exponents, and the precise singular-value scratch
    DevBuf ex_rexp, ex_xd, ex_tr, ex_hi, ex_lo, ex_cexp, ex_yd, ex_tc, ex_svd;
    int64_t ex_ldp = 0, ex_ldy = 0;     // plane and Y-digit leading dimensions
    int ex_cap = 0;                     // width capacity of the exact buffers
    re::BatchedState* batched = nullptr;
    // sketch-size proposal network: parameters, Adam moments, gradient, scratch
    DevBuf mlp_P, mlp_M, mlp_V, mlp_G, mlp_X, mlp_y, mlp_logits, mlp_keep, mlp_cls, mlp_feat, mlp_loss;
    int mlp_step = 0;
    bool mlp_ready = false;
    cudaStream_t copy_stream = nullptr;         // host entry point: chunked copies of A
    std::vector<cudaEvent_t> chunk_events;      // one per copied row chunk (plus the start event)
    re::DevReadoff* h_ro = nullptr;   // pinned
    double* h_sigma = nullptr;        // pinned, 1024 doubles
    int sm_count = 0;
};

namespace re {
int set_last_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace re

namespace {

cudaEvent_t take_event(re_handle h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Stage timing on the caller's stream: begin() returns an event recorded before
// the stage's launches, end() records the closing event.  Timings are resolved
// after the next stream synchronisation.
cudaEvent_t stage_begin(re_handle h, cudaStream_t st) {
    if (!h->timing) return nullptr;
    cudaEvent_t a = take_event(h);
    cudaEventRecord(a, st);
    return a;
}

void stage_end(re_handle h, cudaStream_t st, cudaEvent_t a, int stage, double bytes = 0.0,
               double flops = 0.0) {
    if (!h->timing || !a) return;
    cudaEvent_t b = take_event(h);
    cudaEventRecord(b, st);
    h->pending.push_back(PendingTiming{stage, a, b, bytes, flops});
}

void resolve_timings(re_handle h) {
    for (const PendingTiming& p : h->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.f;
        }
        switch (p.stage) {
            case kStageRight:
                h->stats.right_ms += ms;
                h->stats.right_launches += 1;
                h->stats.right_bytes += p.bytes;
                h->stats.right_flops += p.flops;
                break;
            case kStageLeft: h->stats.left_ms += ms; break;
            case kStageSvd: h->stats.svd_ms += ms; break;
            case kStageQbPre: h->stats.qb_precondition_ms += ms; break;
            case kStageQbOrth: h->stats.qb_orthonormalise_ms += ms; break;
            case kStageQbProduct: h->stats.qb_product_ms += ms; break;
            default: h->stats.other_ms += ms; break;
        }
        h->event_pool.push_back(p.a);
        h->event_pool.push_back(p.b);
    }
    h->pending.clear();
}

int ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.cap) return RE_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(RE_ERR_NOMEM, "device workspace allocation failed");
    }
    b.cap = want;
    return RE_OK;
}

void release(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

int round_half_away_11_10(int r) { return (2 * 11 * r + 10) / 20; }

// r1(s): largest r with round(1.1 r) <= s (Algorithm 1 step 1; 10% oversampling of Sec. 3.3).
int r1_of_s(int s) {
    int r = 1;
    while (round_half_away_11_10(r + 1) <= s) ++r;
    return r;
}

// Left embedding: opts.y_kind, else the right one's kind; the HRTT's is Gaussian
// (the column space of A X is that of A's leading left singular vectors, as
// coherent as A's, where a sampled Hadamard Y aliases).
int left_kind(re_handle h, int kind) {
    if (h->opts.y_kind >= 0) return h->opts.y_kind;
    return kind == RE_HRTT || kind == RE_HRCT ? RE_GAUSSIAN : kind;
}

// Hashed right embeddings (HRTT, HRCT): every column depends on the width, so a
// wider sketch is formed anew from column 0, and the width is at most n_pad.
bool hashed(int kind) { return kind == RE_HRTT || kind == RE_HRCT; }

struct Plan {
    re::MatView A;
    int kind;     // right embedding
    int ykind;    // left embedding
    int cap;      // largest admissible width
    int64_t n_pad, m_pad;
    int nbits, mbits;
};

int make_plan(const void* A, int dtype, int64_t m, int64_t n, int64_t ld, int kind, int ykind,
              int s_max, Plan* p) {
    if (!A) return fail(RE_ERR_ARG, "A is NULL");
    if (dtype != RE_F32 && dtype != RE_F64) return fail(RE_ERR_ARG, "dtype must be RE_F32 or RE_F64");
    if (m <= 0 || n <= 0) return fail(RE_ERR_ARG, "m and n must be positive");
    if (ld < n) return fail(RE_ERR_ARG, "ld < n");
    if (m > INT32_MAX || n > INT32_MAX) return fail(RE_ERR_ARG, "dimension too large");
    if (kind != RE_GAUSSIAN && kind != RE_SRHT && !hashed(kind)) return fail(RE_ERR_ARG, "unknown sketch kind");
    if (ykind != RE_GAUSSIAN && ykind != RE_SRHT && ykind != RE_SRCT) return fail(RE_ERR_ARG, "unknown left sketch kind");
    p->A.ptr = A;
    p->A.dtype = dtype;
    p->A.trans = m < n;
    p->A.rows = std::max(m, n);
    p->A.cols = std::min(m, n);
    p->A.ld = ld;
    p->kind = kind;
    p->ykind = ykind;
    p->nbits = re::pow2_bits(p->A.cols);
    p->mbits = re::pow2_bits(p->A.rows);
    p->n_pad = int64_t(1) << p->nbits;
    p->m_pad = int64_t(1) << p->mbits;
    if (kind != RE_GAUSSIAN && p->nbits > 15)
        return fail(RE_ERR_UNSUPPORTED, "right transforms of more than 2^15 points are not built");
    int64_t cap = s_max;
    if (kind == RE_SRHT || hashed(kind)) cap = std::min<int64_t>(cap, p->n_pad);   // hashed: no empty bucket
    if (ykind == RE_SRHT || ykind == RE_SRCT) cap = std::min<int64_t>(cap, p->m_pad / 2);
    p->cap = (int)cap;
    return RE_OK;
}

// Algorithmic bytes of one right-sketch launch: A read once, X read (x_bytes per
// entry, 0 when generated in place), AX written.
double right_bytes(const Plan& P, int cnt, int x_bytes) {
    const double a_elem = P.A.dtype == RE_F32 ? 4.0 : 8.0;
    return a_elem * (double)P.A.rows * (double)P.A.cols + (double)x_bytes * P.A.cols * cnt +
           4.0 * (double)P.A.rows * cnt;
}

struct Step {
    int passes = 0;
    int final_s = 0;
    re::DevReadoff ro{};
};

// ---- precision mode: exact-product sketches (sketch_ex.cu) ----------------------
bool exact_mode(re_handle h, const Plan& P) { return h->opts.precision == RE_PREC_EXACT && P.kind == RE_GAUSSIAN; }

// Buffers of the exact path for widths up to cap, and the row exponents of A
// (one read of A; Inf/NaN and entries of 2^126 or more are reported here).
int exact_prepare(re_handle h, const Plan& P, int cap, cudaStream_t st) {
    const re::MatView& A = P.A;
    if (A.dtype != RE_F32 || A.trans || (A.ld % 4) != 0 || (reinterpret_cast<uintptr_t>(A.ptr) & 15) != 0)
        return fail(RE_ERR_UNSUPPORTED,
                    "the exact-product precision mode takes FP32 A with m >= n and 16-byte aligned rows");
    if (A.cols > (int64_t(1) << 20)) return fail(RE_ERR_UNSUPPORTED, "the exact-product precision mode takes min(m, n) <= 2^20");
    if (P.ykind != RE_GAUSSIAN) return fail(RE_ERR_UNSUPPORTED, "the exact-product precision mode takes a Gaussian Y");
    const int64_t M = A.rows, Kc = A.cols;
    const int64_t kpad = (Kc + 63) / 64 * 64;
    cap = std::max(cap, 16);
    const int cap16 = (cap + 15) / 16 * 16;
    h->ex_ldp = (M + 3) / 4 * 4;
    h->ex_ldy = (M + 63) / 64 * 64;
    h->ex_cap = cap;
    if (int r = ensure(h->ex_rexp, sizeof(int) * (size_t)M)) return r;
    if (int r = ensure(h->ex_xd, sizeof(uint16_t) * 2 * (size_t)cap16 * kpad)) return r;
    if (int r = ensure(h->ex_tr, sizeof(long long) * (size_t)M * cap)) return r;
    if (int r = ensure(h->ex_hi, sizeof(float) * (size_t)cap * h->ex_ldp)) return r;
    if (int r = ensure(h->ex_lo, sizeof(float) * (size_t)cap * h->ex_ldp)) return r;
    if (int r = ensure(h->ex_cexp, sizeof(int) * (size_t)cap)) return r;
    if (int r = ensure(h->ex_yd, sizeof(uint16_t) * 2 * (size_t)(2 * cap) * h->ex_ldy)) return r;
    if (int r = ensure(h->ex_tc, sizeof(long long) * (size_t)cap * (2 * cap))) return r;
    if (int r = ensure(h->ex_svd, re::svd_precise_bytes(2 * cap, cap))) return r;
    if (int r = ensure(h->status, 64)) return r;
    int* flag = static_cast<int*>(h->status.p) + 4;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    cudaEvent_t g = stage_begin(h, st);
    if (e == cudaSuccess)
        e = re::launch_row_exponent(static_cast<const float*>(A.ptr), A.ld, M, Kc, static_cast<int*>(h->ex_rexp.p),
                                    flag, st);
    stage_end(h, st, g, kStageOther);
    int hf = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "row exponents");
    h->stats.launches += 1;
    if (hf & 1) return fail(RE_ERR_NONFINITE, "non-finite values in A");
    if (hf & 2) return fail(RE_ERR_UNSUPPORTED, "entries of magnitude 2^126 or more are outside the precision mode");
    return RE_OK;
}

// Exact right sketch of columns [c0, c0+cnt): int64 sums, then the FP32 pair planes
// of A X (and, when V is given, its FP64 values) with the column exponents.
int right_columns_exact(re_handle h, const Plan& P, uint64_t seed, int c0, int cnt, double* V, int64_t ldv,
                        cudaStream_t st) {
    const int64_t M = P.A.rows, Kc = P.A.cols, kpad = (Kc + 63) / 64 * 64;
    if (c0 + cnt > h->ex_cap) return fail(RE_ERR_ARG, "exact sketch width exceeds the prepared capacity");
    const int q16 = (cnt + 15) / 16 * 16;
    uint16_t* xd = static_cast<uint16_t*>(h->ex_xd.p);
    long long* T = static_cast<long long*>(h->ex_tr.p);
    int* status = static_cast<int*>(h->status.p);
    cudaEvent_t g = stage_begin(h, st);
    cudaError_t e = re::launch_normal_digits(seed, re::kStreamGX, Kc, kpad, c0, cnt, xd, kpad, q16, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(T, 0, sizeof(long long) * (size_t)M * cnt, st);
    stage_end(h, st, g, kStageOther);
    if (e != cudaSuccess) return cuda_fail(e, "X digits");
    cudaEvent_t a = stage_begin(h, st);
    int nl = 0;
    e = re::launch_ex_sketch(static_cast<const float*>(P.A.ptr), nullptr, P.A.ld, M, Kc,
                             static_cast<const int*>(h->ex_rexp.p), xd, kpad, q16, 0, cnt,
                             reinterpret_cast<unsigned long long*>(T), cnt, status + 1, st, &nl);
    if (e != cudaSuccess) return cuda_fail(e, "right sketch (exact products)");
    stage_end(h, st, a, kStageRight, 4.0 * (double)M * Kc + 4.0 * (double)q16 * Kc + 8.0 * (double)M * cnt,
              9.0 * 2.0 * (double)M * Kc * cnt);
    g = stage_begin(h, st);
    int* cexp = static_cast<int*>(h->ex_cexp.p);
    e = cudaMemsetAsync(cexp + c0, 0x80, sizeof(int) * (size_t)cnt, st);
    if (e == cudaSuccess)
        e = re::launch_ex_finalize(T, cnt, static_cast<const int*>(h->ex_rexp.p), M, cnt,
                                   static_cast<float*>(h->ex_hi.p) + (size_t)c0 * h->ex_ldp,
                                   static_cast<float*>(h->ex_lo.p) + (size_t)c0 * h->ex_ldp, h->ex_ldp, V, ldv,
                                   cexp + c0, st);
    stage_end(h, st, g, kStageOther);
    if (e != cudaSuccess) return cuda_fail(e, "A X from the exact sums");
    h->stats.launches += 3 + nl;
    return RE_OK;
}

// Exact left-sketch blocks after A X columns [c0, c1): Y rows [2 c0, 2 c1) x columns
// [0, c0) and Y rows [0, 2 c1) x columns [c0, c1), FP64 into core.  Y digit rows
// from y_from on are generated (earlier ones are kept from the previous step).
int left_blocks_exact(re_handle h, const Plan& P, uint64_t seed, int c0, int c1, double* core, int64_t ld_core,
                      cudaStream_t st, int y_from) {
    const int64_t M = P.A.rows, ldy = h->ex_ldy, ldp = h->ex_ldp;
    const int slice_rows = 2 * h->ex_cap, ldtc = 2 * h->ex_cap;
    uint16_t* yd = static_cast<uint16_t*>(h->ex_yd.p);
    long long* Tc = static_cast<long long*>(h->ex_tc.p);
    const float* hi = static_cast<const float*>(h->ex_hi.p);
    const float* lo = static_cast<const float*>(h->ex_lo.p);
    const int* cexp = static_cast<const int*>(h->ex_cexp.p);
    int* status = static_cast<int*>(h->status.p);
    cudaEvent_t a = stage_begin(h, st);
    cudaError_t e = re::launch_normal_digits(seed, re::kStreamGY, M, ldy, y_from, 2 * c1 - y_from,
                                             yd + (size_t)y_from * ldy, ldy, slice_rows, st);
    int nl = 1;
    if (e == cudaSuccess && c0 > 0) {
        e = cudaMemset2DAsync(Tc + 2 * c0, sizeof(long long) * ldtc, 0, sizeof(long long) * 2 * (c1 - c0), c0, st);
        if (e == cudaSuccess)
            e = re::launch_ex_sketch(hi, lo, ldp, c0, M, cexp, yd, ldy, slice_rows, 2 * c0, 2 * (c1 - c0),
                                     reinterpret_cast<unsigned long long*>(Tc + 2 * c0), ldtc, status + 1, st, &nl);
        if (e == cudaSuccess)
            e = re::launch_ex_core_finalize(Tc + 2 * c0, ldtc, cexp, c0, 2 * (c1 - c0), 0, 2 * c0, core, ld_core, st);
        ++nl;
    }
    if (e == cudaSuccess)
        e = cudaMemset2DAsync(Tc + (size_t)c0 * ldtc, sizeof(long long) * ldtc, 0, sizeof(long long) * 2 * c1, c1 - c0,
                              st);
    if (e == cudaSuccess)
        e = re::launch_ex_sketch(hi + (size_t)c0 * ldp, lo + (size_t)c0 * ldp, ldp, c1 - c0, M, cexp + c0, yd, ldy,
                                 slice_rows, 0, 2 * c1, reinterpret_cast<unsigned long long*>(Tc + (size_t)c0 * ldtc),
                                 ldtc, status + 1, st, &nl);
    if (e == cudaSuccess)
        e = re::launch_ex_core_finalize(Tc + (size_t)c0 * ldtc, ldtc, cexp, c1 - c0, 2 * c1, c0, 0, core, ld_core, st);
    ++nl;
    if (e != cudaSuccess) return cuda_fail(e, "left sketch (exact products)");
    stage_end(h, st, a, kStageLeft);
    h->stats.launches += nl;
    return RE_OK;
}

// Right sketch columns [c0, c0+cnt) of the oriented A into AX (row-major, ld_ax).
int right_columns(re_handle h, const Plan& P, uint64_t seed, int c0, int cnt, float* AX,
                  int64_t ld_ax, cudaStream_t st) {
    cudaError_t e;
    if (exact_mode(h, P)) return right_columns_exact(h, P, seed, c0, cnt, nullptr, 0, st);
    if (P.kind == RE_GAUSSIAN) {
        // the tensor-core kernel writes AX rows with 16-byte stores
        const bool tc = h->opts.precision == RE_PREC_BF16X3 && re::tc_supported(P.A) && (ld_ax % 4) == 0 &&
                        (reinterpret_cast<uintptr_t>(AX + c0) & 15) == 0;
        if (tc && cnt > 256) {
            // the tensor-core kernel takes at most 256 columns (one MMA N) per pass
            for (int c = 0; c < cnt; c += 256)
                if (int r = right_columns(h, P, seed, c0 + c, std::min(256, cnt - c), AX, ld_ax, st)) return r;
            return RE_OK;
        }
        if (tc) {
            const int64_t kpad = (P.A.cols + 63) / 64 * 64;
            const int nrows = re::tc_mma_n(cnt);
            if (int r = ensure(h->xt, sizeof(uint16_t) * (size_t)kpad * nrows)) return r;
            if (int r = ensure(h->status, 64)) return r;
            cudaEvent_t g = stage_begin(h, st);
            if (nrows > cnt) {
                e = cudaMemsetAsync(static_cast<uint16_t*>(h->xt.p) + (size_t)kpad * cnt, 0,
                                    sizeof(uint16_t) * (size_t)kpad * (nrows - cnt), st);
                if (e != cudaSuccess) return cuda_fail(e, "clear X padding");
            }
            e = re::launch_gauss_xt_bf16(seed, P.A.cols, kpad, c0, cnt, static_cast<uint16_t*>(h->xt.p),
                                         kpad, st);
            if (e != cudaSuccess) return cuda_fail(e, "generate X");
            stage_end(h, st, g, kStageOther);
            cudaEvent_t a = stage_begin(h, st);
            int nl = 0;
            e = re::launch_right_tc(P.A, static_cast<const uint16_t*>(h->xt.p), kpad, cnt,
                                    AX + c0, ld_ax, static_cast<int*>(h->status.p) + 1, st, &nl,
                                    h->opts.test_drop_load);
            if (e != cudaSuccess) return cuda_fail(e, "right sketch (tensor cores)");
            stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 2), 3.0 * 2.0 * P.A.rows * P.A.cols * cnt);
            h->stats.launches += 1 + nl;
            return RE_OK;
        }
        // inputs the tensor-core kernel does not take (transposed or FP64 A,
        // unaligned rows of A or AX) use the FP32 kernel
        if (int r = ensure(h->x, sizeof(float) * (size_t)P.A.cols * cnt)) return r;
        cudaEvent_t g = stage_begin(h, st);
        e = re::launch_gauss_x(seed, P.A.cols, c0, cnt, static_cast<float*>(h->x.p), cnt, st);
        if (e != cudaSuccess) return cuda_fail(e, "generate X");
        stage_end(h, st, g, kStageOther);
        cudaEvent_t a = stage_begin(h, st);
        e = re::launch_right_simt(P.A, static_cast<const float*>(h->x.p), cnt, cnt, AX + c0, ld_ax, st);
        if (e != cudaSuccess) return cuda_fail(e, "right sketch (FP32)");
        stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 4), 2.0 * P.A.rows * P.A.cols * cnt);
        h->stats.launches += 2;
        return RE_OK;
    }
    if (P.kind == RE_HRCT) {
        // hashed randomized DCT of width cnt: X = D F^T C^T generated densely, each entry
        // a compensated FP32 sum over its bucket's scaled cosines (columns depend on
        // the width: c0 is where AX receives them)
        if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)(P.n_pad / 32 + 1))) return r;
        if (int r = ensure(h->ht, sizeof(uint16_t) * (size_t)P.n_pad)) return r;
        if (int r = ensure(h->ctabx, sizeof(float) * (size_t)(P.n_pad + 1))) return r;
        if (int r = ensure(h->status, 64)) return r;
        cudaEvent_t g = stage_begin(h, st);
        e = re::launch_sign_bits(seed, re::kStreamDX, P.A.cols, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_hrtt_table(seed, P.nbits, static_cast<uint16_t*>(h->ht.p), st);
        if (e == cudaSuccess) e = re::launch_cos_table(P.nbits, static_cast<float*>(h->ctabx.p), st);
        stage_end(h, st, g, kStageOther);
        if (e != cudaSuccess) return cuda_fail(e, "generate X (HRCT)");
        h->stats.launches += 3;
        const uint32_t* dx = static_cast<const uint32_t*>(h->dx.p);
        const uint16_t* tbl = static_cast<const uint16_t*>(h->ht.p);
        const float* ctab = static_cast<const float*>(h->ctabx.p);
        const bool tc = h->opts.precision == RE_PREC_BF16X3 && re::tc_supported(P.A) && (ld_ax % 4) == 0 &&
                        (reinterpret_cast<uintptr_t>(AX + c0) & 15) == 0;
        if (tc) {
            // the FP32 X as its three exact BF16 terms: six products per K step, 128
            // columns per launch (shared memory holds three planes of 128 rows)
            const int64_t kpad = (P.A.cols + 63) / 64 * 64;
            for (int j0 = 0; j0 < cnt; j0 += 128) {
                const int w = std::min(128, cnt - j0);
                const int nrows = re::tc_mma_n(w);
                if (int r = ensure(h->xt, sizeof(uint16_t) * (size_t)kpad * nrows * 3)) return r;
                cudaEvent_t g2 = stage_begin(h, st);
                for (int pl = 0; pl < 3 && e == cudaSuccess && nrows > w; ++pl)
                    e = cudaMemsetAsync(static_cast<uint16_t*>(h->xt.p) + (size_t)kpad * ((size_t)pl * nrows + w), 0,
                                        sizeof(uint16_t) * (size_t)kpad * (nrows - w), st);
                if (e == cudaSuccess)
                    e = re::launch_hrct_x(P.A.cols, kpad, cnt, j0, w, P.nbits, dx, tbl, ctab, 3, nullptr,
                                          static_cast<uint16_t*>(h->xt.p), kpad, nrows, st);
                stage_end(h, st, g2, kStageOther);
                if (e != cudaSuccess) return cuda_fail(e, "generate X (HRCT)");
                cudaEvent_t a2 = stage_begin(h, st);
                int nl = 0;
                e = re::launch_right_tc(P.A, static_cast<const uint16_t*>(h->xt.p), kpad, w, AX + c0 + j0, ld_ax,
                                        static_cast<int*>(h->status.p) + 1, st, &nl, h->opts.test_drop_load, 3);
                if (e != cudaSuccess) return cuda_fail(e, "right sketch (HRCT, tensor cores)");
                stage_end(h, st, a2, kStageRight, right_bytes(P, w, 6), 6.0 * 2.0 * P.A.rows * P.A.cols * w);
                h->stats.launches += 1 + nl;
            }
            return RE_OK;
        }
        if (int r = ensure(h->x, sizeof(float) * (size_t)P.A.cols * cnt)) return r;
        cudaEvent_t g2 = stage_begin(h, st);
        e = re::launch_hrct_x(P.A.cols, 0, cnt, 0, cnt, P.nbits, dx, tbl, ctab, 0, static_cast<float*>(h->x.p),
                              nullptr, cnt, 0, st);
        stage_end(h, st, g2, kStageOther);
        if (e != cudaSuccess) return cuda_fail(e, "generate X (HRCT)");
        cudaEvent_t a = stage_begin(h, st);
        e = re::launch_right_simt(P.A, static_cast<const float*>(h->x.p), cnt, cnt, AX + c0, ld_ax, st);
        if (e != cudaSuccess) return cuda_fail(e, "right sketch (HRCT, FP32)");
        stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 4), 2.0 * P.A.rows * P.A.cols * cnt);
        h->stats.launches += 2;
        return RE_OK;
    }
    if (P.kind == RE_HRTT) {
        // HRTT of width cnt (columns depend on the width: c0 is where AX receives them)
        if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)(P.n_pad / 32 + 1))) return r;
        if (int r = ensure(h->ht, sizeof(uint16_t) * (size_t)P.n_pad)) return r;
        cudaEvent_t g = stage_begin(h, st);
        e = re::launch_sign_bits(seed, re::kStreamDX, P.A.cols, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_hrtt_table(seed, P.nbits, static_cast<uint16_t*>(h->ht.p), st);
        stage_end(h, st, g, kStageOther);
        if (int r = ensure(h->status, 64)) return r;
        const bool tc = h->opts.precision == RE_PREC_BF16X3 && re::tc_supported(P.A) && (ld_ax % 4) == 0 &&
                        (reinterpret_cast<uintptr_t>(AX + c0) & 15) == 0;
        if (e == cudaSuccess && tc) {
            // the dense X = D H C^T has integer entries of magnitude at most the bucket
            // size: exact in BF16 when buckets hold at most 256 coordinates (one plane,
            // 256 columns per launch), otherwise as a BF16 and its remainder (two planes,
            // six products, 128 columns per launch); the width goes through the
            // tensor-core contraction instead of the register transform
            const int planes = P.n_pad <= 256 * (int64_t)cnt ? 1 : 2;
            const int wmax = planes == 1 ? 256 : 128;
            const int64_t kpad = (P.A.cols + 63) / 64 * 64;
            for (int j0 = 0; j0 < cnt && e == cudaSuccess; j0 += wmax) {
                const int w = std::min(wmax, cnt - j0);
                const int nrows = re::tc_mma_n(w);
                if (int r = ensure(h->xt, sizeof(uint16_t) * (size_t)kpad * nrows * planes)) return r;
                cudaEvent_t g2 = stage_begin(h, st);
                for (int pl = 0; pl < planes && e == cudaSuccess && nrows > w; ++pl)
                    e = cudaMemsetAsync(static_cast<uint16_t*>(h->xt.p) + (size_t)kpad * ((size_t)pl * nrows + w), 0,
                                        sizeof(uint16_t) * (size_t)kpad * (nrows - w), st);
                if (e == cudaSuccess)
                    e = re::launch_hrtt_xt_bf16(P.A.cols, kpad, cnt, j0, w, P.nbits,
                                                static_cast<const uint32_t*>(h->dx.p),
                                                static_cast<const uint16_t*>(h->ht.p),
                                                static_cast<uint16_t*>(h->xt.p), kpad, st, planes, nrows);
                stage_end(h, st, g2, kStageOther);
                if (e != cudaSuccess) break;
                cudaEvent_t a2 = stage_begin(h, st);
                int nl = 0;
                e = re::launch_right_tc(P.A, static_cast<const uint16_t*>(h->xt.p), kpad, w, AX + c0 + j0, ld_ax,
                                        static_cast<int*>(h->status.p) + 1, st, &nl, h->opts.test_drop_load, planes);
                stage_end(h, st, a2, kStageRight, right_bytes(P, w, 2 * planes),
                          3.0 * planes * 2.0 * P.A.rows * P.A.cols * w);
                h->stats.launches += 1 + nl;
            }
            if (e != cudaSuccess) return cuda_fail(e, "right sketch (HRTT, tensor cores)");
            h->stats.launches += 2;
            return RE_OK;
        }
        cudaEvent_t a = stage_begin(h, st);
        if (e == cudaSuccess)
            e = re::launch_right_hrtt(P.A, static_cast<const uint32_t*>(h->dx.p), static_cast<uint16_t*>(h->ht.p),
                                      cnt, AX + c0, ld_ax, st, static_cast<int*>(h->status.p) + 1);
        if (e != cudaSuccess) return cuda_fail(e, "right sketch (HRTT)");
        stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 0),
                  (double)P.A.rows * (double)P.n_pad * (double)(P.nbits + 1));
        h->stats.launches += 3;
        return RE_OK;
    }
    // SRHT: signs of the padded n and sampled columns pi_X(c0 .. c0+cnt-1)
    if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)(P.n_pad / 32 + 1))) return r;
    if (int r = ensure(h->px, sizeof(int) * (size_t)cnt)) return r;
    const bool tc = h->opts.precision == RE_PREC_BF16X3 && re::tc_supported(P.A) && (ld_ax % 4) == 0 &&
                    (reinterpret_cast<uintptr_t>(AX + c0) & 15) == 0;
    if (tc && cnt > 256) {
        for (int c = 0; c < cnt; c += 256)
            if (int r = right_columns(h, P, seed, c0 + c, std::min(256, cnt - c), AX, ld_ax, st)) return r;
        return RE_OK;
    }
    if (tc) {
        // X = D H S^T has +-1 entries, exact in BF16: the sampled columns go through the
        // tensor-core contraction of the Gaussian sketch (A in three BF16 terms, exact
        // products, FP32 accumulation) instead of the register transform
        const int64_t kpad = (P.A.cols + 63) / 64 * 64;
        const int nrows = re::tc_mma_n(cnt);
        if (int r = ensure(h->xt, sizeof(uint16_t) * (size_t)kpad * nrows)) return r;
        if (int r = ensure(h->status, 64)) return r;
        cudaEvent_t g = stage_begin(h, st);
        e = re::launch_sign_bits(seed, re::kStreamDX, P.A.cols, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_perm(seed, re::kStreamPX, P.nbits, c0, cnt, static_cast<int*>(h->px.p), st);
        if (e == cudaSuccess && nrows > cnt)
            e = cudaMemsetAsync(static_cast<uint16_t*>(h->xt.p) + (size_t)kpad * cnt, 0,
                                sizeof(uint16_t) * (size_t)kpad * (nrows - cnt), st);
        if (e == cudaSuccess)
            e = re::launch_srht_xt_bf16(P.A.cols, kpad, static_cast<const int*>(h->px.p),
                                        static_cast<const uint32_t*>(h->dx.p), cnt, static_cast<uint16_t*>(h->xt.p),
                                        kpad, st);
        if (e != cudaSuccess) return cuda_fail(e, "generate X (SRHT)");
        stage_end(h, st, g, kStageOther);
        cudaEvent_t a = stage_begin(h, st);
        int nl = 0;
        e = re::launch_right_tc(P.A, static_cast<const uint16_t*>(h->xt.p), kpad, cnt, AX + c0, ld_ax,
                                static_cast<int*>(h->status.p) + 1, st, &nl, h->opts.test_drop_load);
        if (e != cudaSuccess) return cuda_fail(e, "right sketch (SRHT, tensor cores)");
        stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 2), 3.0 * 2.0 * P.A.rows * P.A.cols * cnt);
        h->stats.launches += 3 + nl;
        return RE_OK;
    }
    cudaEvent_t g = stage_begin(h, st);
    e = re::launch_sign_bits(seed, re::kStreamDX, P.A.cols, static_cast<uint32_t*>(h->dx.p), st);
    if (e == cudaSuccess)
        e = re::launch_perm(seed, re::kStreamPX, P.nbits, c0, cnt, static_cast<int*>(h->px.p), st);
    stage_end(h, st, g, kStageOther);
    if (int r = ensure(h->status, 64)) return r;
    cudaEvent_t a = stage_begin(h, st);
    if (e == cudaSuccess)
        e = re::launch_right_srht(P.A, static_cast<const uint32_t*>(h->dx.p),
                                  static_cast<const int*>(h->px.p), cnt, AX + c0, ld_ax, st,
                                  static_cast<int*>(h->status.p) + 1);
    if (e != cudaSuccess) return cuda_fail(e, "right sketch (SRHT)");
    stage_end(h, st, a, kStageRight, right_bytes(P, cnt, 0),
              (double)P.A.rows * (double)P.n_pad * (double)P.nbits);
    h->stats.launches += 3;
    return RE_OK;
}

// Left-sketch blocks after AX columns [c0, c1) were added: rows [2 c0, 2 c1) x cols
// [0, c0) and rows [0, 2 c1) x cols [c0, c1) of core (FP64 row-major, ld_core).
// With the SRTT Y the columns are transformed once into the handle's Z (H D AX,
// m_pad x ld_ax) and the blocks sampled from it: within one estimate only the new
// columns are transformed (transform_from = c0); a standalone sketch step
// transforms from column 0 (the caller supplies the earlier AX columns).
int left_blocks(re_handle h, const Plan& P, uint64_t seed, int c0, int c1, const float* AX,
                int64_t ld_ax, double* core, int64_t ld_core, cudaStream_t st, int transform_from) {
    if (exact_mode(h, P)) return left_blocks_exact(h, P, seed, c0, c1, core, ld_core, st, 2 * c0);
    const int64_t M = P.A.rows;
    if (int r = ensure(h->status, 64)) return r;
    if (P.ykind == RE_SRHT) {
        if (int r = ensure(h->dy, sizeof(uint32_t) * (size_t)(P.m_pad / 32 + 1))) return r;
        if (int r = ensure(h->py, sizeof(int) * (size_t)(2 * c1))) return r;
        if (int r = ensure(h->fz, sizeof(float) * (size_t)P.m_pad * (size_t)ld_ax)) return r;
        cudaEvent_t g = stage_begin(h, st);
        cudaError_t e = re::launch_sign_bits(seed, re::kStreamDY, M, static_cast<uint32_t*>(h->dy.p), st);
        if (e == cudaSuccess)
            e = re::launch_perm(seed, re::kStreamPY, P.mbits, 0, 2 * c1, static_cast<int*>(h->py.p), st);
        if (e != cudaSuccess) return cuda_fail(e, "left embedding");
        stage_end(h, st, g, kStageOther);
        float* Z = static_cast<float*>(h->fz.p);
        const int* perm = static_cast<const int*>(h->py.p);
        cudaEvent_t a = stage_begin(h, st);
        e = re::launch_left_srtt_transform(AX, ld_ax, M, P.mbits, static_cast<const uint32_t*>(h->dy.p),
                                           transform_from, c1, Z, ld_ax, st);
        if (e == cudaSuccess && c0 > 0)
            e = re::launch_left_srtt_sample(Z, ld_ax, perm, 2 * c0, 2 * (c1 - c0), 0, c0, core, ld_core, st);
        if (e == cudaSuccess) e = re::launch_left_srtt_sample(Z, ld_ax, perm, 0, 2 * c1, c0, c1 - c0, core, ld_core, st);
        if (e != cudaSuccess) return cuda_fail(e, "left sketch (SRTT)");
        stage_end(h, st, a, kStageLeft);
        h->stats.launches += 2 + (P.mbits + 9) / 10 + (c0 > 0 ? 2 : 1);
        return RE_OK;
    }
    if (P.ykind == RE_SRCT) {
        // DCT rows generated inside the CUDA-core left kernel from the sampled
        // frequencies, the signs and a cosine table of the padded order
        if (int r = ensure(h->dy, sizeof(uint32_t) * (size_t)(P.m_pad / 32 + 1))) return r;
        if (int r = ensure(h->py, sizeof(int) * (size_t)(2 * c1))) return r;
        if (int r = ensure(h->ctab, sizeof(float) * (size_t)(P.m_pad + 1))) return r;
        const size_t needc = std::max({re::left_part_floats(M, 2 * (c1 - c0), c0),
                                       re::left_part_floats(M, 2 * c1, c1 - c0),
                                       re::left_tc_part_floats(M, 2 * (c1 - c0), c0, true),
                                       re::left_tc_part_floats(M, 2 * c1, c1 - c0, true)});
        if (int r = ensure(h->part, sizeof(float) * needc)) return r;
        if (int r = ensure(h->status, 64)) return r;
        int* tmo = static_cast<int*>(h->status.p) + 1;   // bounded-wait expiry flag of the tensor-core kernels
        cudaEvent_t g = stage_begin(h, st);
        cudaError_t e = re::launch_sign_bits(seed, re::kStreamDY, M, static_cast<uint32_t*>(h->dy.p), st);
        if (e == cudaSuccess)
            e = re::launch_perm(seed, re::kStreamPY, P.mbits, 0, 2 * c1, static_cast<int*>(h->py.p), st);
        if (e == cudaSuccess) e = re::launch_cos_table(P.mbits, static_cast<float*>(h->ctab.p), st);
        if (e != cudaSuccess) return cuda_fail(e, "left embedding");
        stage_end(h, st, g, kStageOther);
        re::DctRows Yd{static_cast<const int*>(h->py.p), static_cast<const uint32_t*>(h->dy.p),
                       static_cast<const float*>(h->ctab.p), P.mbits};
        cudaEvent_t a = stage_begin(h, st);
        float* part = static_cast<float*>(h->part.p);
        const size_t cap = h->part.cap / sizeof(float);
        // on the tensor cores when AX is aligned (Y and AX as three exact BF16 terms
        // each, six products, FP32 accumulation: the numerics of an FP32 product, as
        // for the Gaussian Y), else on CUDA cores
        int* tflag = tmo;
        if (c0 > 0)
            e = re::launch_left_dct(Yd, AX, ld_ax, M, 2 * c0, 2 * (c1 - c0), 0, c0, part, cap, core, ld_core, st,
                                    tflag);
        if (e == cudaSuccess)
            e = re::launch_left_dct(Yd, AX, ld_ax, M, 0, 2 * c1, c0, c1 - c0, part, cap, core, ld_core, st, tflag);
        if (e != cudaSuccess) return cuda_fail(e, "left sketch (SRCT)");
        stage_end(h, st, a, kStageLeft);
        h->stats.launches += 3 + (c0 > 0 ? 4 : 2);
        return RE_OK;
    }
    // the new core entries as two rectangles that each need their own Y rows once:
    // rows [2 c0, 2 c1) x columns [0, c1) and rows [0, 2 c0) x columns [c0, c1) (the
    // Gaussian Y is generated inside the kernels, and generating it is what they spend
    // their time on)
    const size_t need = std::max({re::left_part_floats(M, 2 * (c1 - c0), c1),
                                  re::left_part_floats(M, 2 * c0, c1 - c0),
                                  re::left_tc_part_floats(M, 2 * (c1 - c0), c1),
                                  re::left_tc_part_floats(M, 2 * c0, c1 - c0)});
    if (int r = ensure(h->part, sizeof(float) * need)) return r;
    int* tmo = static_cast<int*>(h->status.p) + 1;     // bounded-wait expiry flag of the tensor-core kernels
    cudaError_t e = cudaSuccess;
    cudaEvent_t a = stage_begin(h, st);
    e = re::launch_left(seed, AX, ld_ax, M, 2 * c0, 2 * (c1 - c0), 0, c1, static_cast<float*>(h->part.p),
                        h->part.cap / sizeof(float), core, ld_core, st, tmo);
    if (e == cudaSuccess && c0 > 0)
        e = re::launch_left(seed, AX, ld_ax, M, 0, 2 * c0, c0, c1 - c0, static_cast<float*>(h->part.p),
                            h->part.cap / sizeof(float), core, ld_core, st, tmo);
    if (e != cudaSuccess) return cuda_fail(e, "left sketch");
    stage_end(h, st, a, kStageLeft);
    h->stats.launches += c0 > 0 ? 4 : 2;
    return RE_OK;
}

// Singular values and read-off of the leading 2s x s block of the core (the
// core at width s, by the nested-prefix property of the appended embeddings).
int check_width(re_handle h, const Plan& P, int s, int smax, double eps, re::DevReadoff* ro, int* r1_out,
                cudaStream_t st, bool may_skip = false) {
    double* core = static_cast<double*>(h->core.p);
    int* status = static_cast<int*>(h->status.p);
    const int r1c = std::min(r1_of_s(s), s);
    // at widths that are not the last, a certified "not converged" skips the
    // Jacobi sweeps; the margin 4 max(eps, 1e-5) keeps the decision clear of the
    // FP32 sweeps' absolute error (about 3e-5 sigma_1), and ||A|| from opts is
    // not used there (the certificate compares with sigma_1 of the core)
    const bool skip_ok = may_skip && h->opts.norm_a <= 0.0 && r1c < P.A.cols;
    const float ratio = (float)(4.0 * std::max(eps, 1e-5));
    const int r1 = std::min(r1_of_s(s), s);
    // X = G/sqrt(s) or D H S^T/sqrt(s); the hashed forms' D (F/sqrt(n_pad)) C^T with F the
    // Hadamard or the scaled DCT-II; Y scaled by 1/sqrt(2s)
    const double xs = hashed(P.kind) ? (double)P.n_pad : (double)s;
    const double scale = 1.0 / std::sqrt(xs * (double)(2 * s));
    // the precision mode takes the preconditioned FP32 singular values (stage 1 is
    // the plain FP32 step, which may first certify that this width cannot succeed)
    const bool precise = exact_mode(h, P);
    bool certify = skip_ok;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = cudaMemsetAsync(status + 3, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "clear status");
        cudaEvent_t a = stage_begin(h, st);
        if (h->opts.sigma_est == RE_SIGMA_QRDIAG)
            e = re::launch_core_qrdiag(core, 2 * s, s, smax, h->svdws.p, static_cast<double*>(h->sigma.p), status, st);
        else if (precise && !(certify && re::core_sigma_fits_cta(2 * s, s)))
            e = re::launch_core_sigma_precise(core, 2 * s, s, smax, h->svdws.p, h->ex_svd.p,
                                              static_cast<double*>(h->sigma.p), status, st);
        else
            e = re::launch_core_sigma(core, 2 * s, s, smax, h->svdws.p, static_cast<double*>(h->sigma.p), status, st,
                                      skip_ok ? r1c : 0, ratio);
        if (e != cudaSuccess) return cuda_fail(e, "core singular values");
        stage_end(h, st, a, kStageSvd);
        e = re::launch_readoff(static_cast<const double*>(h->sigma.p), r1, scale, eps, h->opts.norm_a, status,
                               static_cast<re::DevReadoff*>(h->ro.p), static_cast<double*>(h->sigma_scaled.p), st);
        if (e != cudaSuccess) return cuda_fail(e, "read-off");
        e = cudaMemcpyAsync(h->h_ro, h->ro.p, sizeof(re::DevReadoff), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "read-off copy");
        h->stats.launches += 2;
        resolve_timings(h);
        // a certified width (no Jacobi, tau = 0) needs nothing more; otherwise the
        // precision mode replaces the FP32 values by the preconditioned ones
        const bool certified = h->h_ro->rank < 0 && h->h_ro->sweeps == 0 && h->h_ro->tau == 0.0;
        if (!precise || !certify || certified || h->h_ro->status != RE_OK ||
            !re::core_sigma_fits_cta(2 * s, s))
            break;
        certify = false;
    }
    *ro = *h->h_ro;
    *r1_out = r1;
    if (ro->status == RE_ERR_TIMEOUT) return fail(ro->status, "a bounded device wait expired");
    if (ro->status != RE_OK) return fail(ro->status, "non-finite values in A or its sketch");
    return RE_OK;
}

// Proposal network: class of the width at which the read-off is expected to
// succeed, from the trusted sigma of the s = 16 core (sigma_scaled).
int propose_width(re_handle h, const Plan& P, double eps, int* cls, cudaStream_t st) {
    if (int r = ensure(h->mlp_feat, sizeof(float) * re::kMlpIn)) return r;
    if (int r = ensure(h->mlp_logits, sizeof(float) * re::kMlpOut)) return r;
    if (int r = ensure(h->mlp_cls, sizeof(int))) return r;
    cudaError_t e = re::mlp_features(static_cast<const double*>(h->sigma_scaled.p), eps, P.A.rows, P.A.cols,
                                     static_cast<float*>(h->mlp_feat.p), st);
    if (e == cudaSuccess)
        e = re::mlp_forward(static_cast<const float*>(h->mlp_P.p), static_cast<const float*>(h->mlp_feat.p), 1,
                            static_cast<float*>(h->mlp_logits.p), nullptr, st);
    if (e == cudaSuccess) e = re::mlp_argmax(static_cast<const float*>(h->mlp_logits.p), 1, static_cast<int*>(h->mlp_cls.p), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cls, h->mlp_cls.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "proposal network");
    h->stats.launches += 3;
    return RE_OK;
}

// Algorithm 1 with doubling on an already validated plan.  With the proposal
// network enabled, the first pass goes straight to s = 16, the network picks a
// target width s*, one more pass appends up to s*, and the read-off is checked
// on the nested leading blocks at every ladder width up to s* in order -- so the
// answer is the plain ladder's whenever s* is at least the plain final width;
// otherwise doubling continues from s*.  The HRTT's columns depend on the
// width, so with it every step sketches A and forms the core anew.
// pre > 0: the caller has already written columns [0, pre) of the handle's AX
// (first pass of the host entry point); the first pass then only adds the core.
int run_estimate(re_handle h, const Plan& P, double eps, uint64_t seed, double* sigma_out, int sigma_cap,
                 re_result* out, cudaStream_t st, int pre = 0) {
    const re_opts& o = h->opts;
    if (o.s0 > P.cap) return fail(RE_ERR_ARG, "initial sketch width exceeds the admissible width");
    if (o.learned && !h->mlp_ready) return fail(RE_ERR_ARG, "learned proposal requested but no network is loaded");
    if (o.learned && hashed(P.kind))
        return fail(RE_ERR_UNSUPPORTED, "the proposal network needs an appendable embedding (Gaussian or SRHT)");
    int smax = o.s0;
    while (smax * 2 <= P.cap) smax *= 2;
    const int64_t M = P.A.rows;
    if (int r = ensure(h->ax, sizeof(float) * (size_t)M * smax)) return r;
    if (int r = ensure(h->core, sizeof(double) * (size_t)2 * smax * smax)) return r;
    if (int r = ensure(h->sigma, sizeof(double) * (size_t)smax)) return r;
    if (int r = ensure(h->sigma_scaled, sizeof(double) * (size_t)smax)) return r;
    if (int r = ensure(h->svdws, re::svd_workspace_bytes(2 * smax, smax))) return r;
    if (int r = ensure(h->ro, sizeof(re::DevReadoff))) return r;
    if (int r = ensure(h->status, 64)) return r;
    float* AX = static_cast<float*>(h->ax.p);
    double* core = static_cast<double*>(h->core.p);
    {
        cudaError_t e0 = cudaMemsetAsync(h->status.p, 0, 4 * sizeof(int), st);
        if (e0 != cudaSuccess) return cuda_fail(e0, "clear status");
    }
    if (exact_mode(h, P)) {
        if (int r = exact_prepare(h, P, smax, st)) return r;
    }
    auto sketch_to = [&](int c0, int c1) -> int {
        if (int r = right_columns(h, P, seed, c0, c1 - c0, AX, smax, st)) return r;
        if (int r = left_blocks(h, P, seed, c0, c1, AX, smax, core, smax, st, c0)) return r;
        h->stats.passes += 1;
        return RE_OK;
    };
    int s_prev = 0, s = o.s0, passes = 0, r1 = 0;
    re::DevReadoff ro{};
    bool done = false;
    if (o.learned && o.s0 == 8 && smax >= 16) {
        if (int r = sketch_to(0, 16)) return r;
        passes = 1;
        for (int w = 8; w <= 16 && !done; w *= 2) {
            if (int r = check_width(h, P, w, smax, eps, &ro, &r1, st, 2 * w <= smax)) return r;
            s = w;
            done = ro.rank >= 0 || r1 >= P.A.cols;
        }
        if (!done && smax >= 32) {
            int cls = 0;
            if (int r = propose_width(h, P, eps, &cls, st)) return r;
            const int target = std::min(smax, std::max(32, 8 << std::min(std::max(cls, 0), 11)));
            // one pass appends the right sketch up to the proposed width; the core
            // is extended one ladder width at a time, only as far as the checks go
            if (int r = right_columns(h, P, seed, 16, target - 16, AX, smax, st)) return r;
            h->stats.passes += 1;
            passes = 2;
            for (int w = 32; w <= target && !done; w *= 2) {
                if (int r = left_blocks(h, P, seed, w / 2, w, AX, smax, core, smax, st, w / 2)) return r;
                if (int r = check_width(h, P, w, smax, eps, &ro, &r1, st, 2 * w <= smax)) return r;
                s = w;
                done = ro.rank >= 0 || r1 >= P.A.cols;
            }
        }
        if (!done) {
            if (2 * s > smax) {
                done = true;          // ladder exhausted at s: r1(s) is a lower bound
            } else {
                s_prev = s;
                s *= 2;
            }
        }
    }
    // The exact-product sketch costs about the same per pass for up to 64 new columns
    // (one Q tile: its MMA count does not depend on the tile's width), so its first
    // pass appends up to 64 columns at once and the read-off runs on the nested
    // leading blocks of the core at s0, 2 s0, ... within it: the plain ladder's
    // answer, with fewer passes over A.  The FP32 and BF16x3 Gaussian ladders do
    // the same up to opts.first_width (HBM-bound passes cost the same for 8 or 128
    // columns), and up to `pre` when the caller sketched that far.
    int wfirst = 0;
    if (exact_mode(h, P)) wfirst = 64;
    else if (P.kind == RE_GAUSSIAN) wfirst = std::max(pre, o.first_width);
    if (!done && !o.learned && wfirst > 0 && s_prev == 0) {
        int w1 = s;
        while (w1 * 2 <= std::min(wfirst, smax)) w1 *= 2;
        if (w1 > s || pre > 0) {
            if (pre >= w1) {
                if (int r = left_blocks(h, P, seed, 0, w1, AX, smax, core, smax, st, 0)) return r;
                h->stats.passes += 1;
            } else if (int r = sketch_to(0, w1)) {
                return r;
            }
            passes = 1;
            for (int w = s; w <= w1 && !done; w *= 2) {
                if (int r = check_width(h, P, w, smax, eps, &ro, &r1, st, 2 * w <= smax)) return r;
                s = w;
                done = ro.rank >= 0 || r1 >= P.A.cols;
            }
            if (!done) {
                if (2 * s > smax) {
                    done = true;
                } else {
                    s_prev = s;
                    s *= 2;
                }
            }
        }
    }
    while (!done) {
        if (int r = sketch_to(hashed(P.kind) ? 0 : s_prev, s)) return r;
        ++passes;
        if (int r = check_width(h, P, s, smax, eps, &ro, &r1, st, 2 * s <= smax)) return r;
        if (ro.rank >= 0 || 2 * s > smax || r1 >= P.A.cols) break;
        s_prev = s;
        s *= 2;
    }
    const int ncopy = std::min(r1, std::max(sigma_cap, 0));
    if (sigma_out && ncopy > 0) {
        cudaError_t e = cudaMemcpyAsync(sigma_out, h->sigma_scaled.p, sizeof(double) * ncopy,
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "sigma copy");
    }
    std::memset(out, 0, sizeof(*out));
    const bool conv = ro.rank >= 0;
    out->rank = conv ? ro.rank : r1;
    out->gap_index = ro.gap_index;
    out->gap_ratio = ro.gap_ratio;
    out->tau = ro.tau;
    out->n_sigma = r1;
    out->final_s = s;
    out->passes = passes;
    out->flags = (conv ? RE_CONVERGED : RE_LOWER_BOUND_ONLY) | (P.A.trans ? RE_TRANSPOSED : 0u);
    out->status = RE_OK;
    out->svd_sweeps = ro.sweeps;
    return RE_OK;
}

// Algorithm 3 (Sec. 5.1): the doubling ladder of Algorithm 1 with the Frobenius
// criterion of step 5 as its stopping rule, then the thin QR of the first
// k = r + p columns of A X and B = Q^T A (rangefinder.cu).
int run_qb(re_handle h, const Plan& P, double eps, int p, uint64_t seed, float* Q, int64_t ldq, float* B,
           int64_t ldb, int k_cap, re_qb_result* out, cudaStream_t st) {
    const re_opts& o = h->opts;
    const bool exact = exact_mode(h, P);
    if (o.s0 > P.cap) return fail(RE_ERR_ARG, "initial sketch width exceeds the admissible width");
    int smax = o.s0;
    while (smax * 2 <= P.cap) smax *= 2;
    const int64_t M = P.A.rows;
    if (int r = ensure(h->ax, sizeof(float) * (size_t)M * smax)) return r;
    if (int r = ensure(h->core, sizeof(double) * (size_t)2 * smax * smax)) return r;
    if (int r = ensure(h->sigma, sizeof(double) * (size_t)smax)) return r;
    if (int r = ensure(h->sigma_scaled, sizeof(double) * (size_t)smax)) return r;
    if (int r = ensure(h->svdws, re::svd_workspace_bytes(2 * smax, smax))) return r;
    if (int r = ensure(h->ro, sizeof(re::DevReadoff))) return r;
    if (int r = ensure(h->status, 64)) return r;
    if (int r = ensure(h->qbsel, sizeof(re::QbSelect) + 16)) return r;
    float* AX = static_cast<float*>(h->ax.p);
    double* core = static_cast<double*>(h->core.p);
    re::QbSelect* sel_dev = static_cast<re::QbSelect*>(h->qbsel.p);
    int* floored = reinterpret_cast<int*>(static_cast<char*>(h->qbsel.p) + sizeof(re::QbSelect));
    cudaError_t e = cudaMemsetAsync(h->status.p, 0, 4 * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(floored, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    // the exact-product sketch resolves the tail values that step 5 sums (its A X
    // stays in FP32 pair planes; the factorization takes their leading FP32 part)
    if (exact) {
        if (int r = exact_prepare(h, P, smax, st)) return r;
    }
    std::memset(out, 0, sizeof(*out));
    int s_prev = 0, s = o.s0, passes = 0, r1 = 0;
    re::DevReadoff ro{};
    re::QbSelect sel{};
    for (;;) {
        if (int r = right_columns(h, P, seed, s_prev, s - s_prev, AX, smax, st)) return r;
        if (int r = left_blocks(h, P, seed, s_prev, s, AX, smax, core, smax, st, s_prev)) return r;
        h->stats.passes += 1;
        ++passes;
        if (int r = check_width(h, P, s, smax, eps, &ro, &r1, st, false)) {
            out->status = r;
            return r;
        }
        e = re::launch_select_rank(static_cast<const double*>(h->sigma_scaled.p), r1, P.A.cols, eps, o.norm_a, p,
                                   s, sel_dev, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&sel, sel_dev, sizeof(sel), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "rank selection");
        h->stats.launches += 1;
        if (sel.met || 2 * s > smax || r1 >= P.A.cols) break;
        s_prev = s;
        s *= 2;
    }
    const bool met = sel.met != 0;
    const int k = (int)std::min<int64_t>(met ? sel.r + p : s, P.A.cols);
    const int r = met ? sel.r : std::max(k - p, 0);
    out->r = r;
    out->k = k;
    out->final_s = s;
    out->passes = passes;
    out->flags = (met ? RE_CONVERGED : RE_LOWER_BOUND_ONLY) | (P.A.trans ? RE_TRANSPOSED : 0u);
    out->bound = met ? sel.bound : -1.0;
    out->norm_a = sel.norm_a;
    if (k > k_cap) return fail(RE_ERR_ARG, "k_cap is smaller than the chosen k = r + p (out->k holds it)");
    if (ldq < k) return fail(RE_ERR_ARG, "ldq < k");
    // B = Q^T A on the tensor cores (BF16x3 split of both factors) unless the
    // handle asks for the plain FP32 form
    const bool tensor = o.precision == RE_PREC_BF16X3 || exact;
    if (int rr = ensure(h->qbws, re::qb_workspace_bytes(M, P.A.cols, k, tensor))) return rr;
    int nl = 0;
    cudaEvent_t a = stage_begin(h, st);
    int* tmo_flag = static_cast<int*>(h->status.p) + 1;   // bounded-wait expiry of the tensor-core kernels
    e = exact ? re::launch_qb_precondition(static_cast<const float*>(h->ex_hi.p), 1, h->ex_ldp, M, P.A.cols, core,
                                           smax, 2 * s, k, h->qbws.p, floored, st, &nl, tensor, tmo_flag)
              : re::launch_qb_precondition(AX, smax, 1, M, P.A.cols, core, smax, 2 * s, k, h->qbws.p, floored, st,
                                           &nl, tensor, tmo_flag);
    stage_end(h, st, a, kStageQbPre);
    if (e == cudaSuccess) {
        a = stage_begin(h, st);
        e = re::launch_qb_orthonormalise(M, P.A.cols, k, Q, ldq, h->qbws.p, floored, st, &nl, tensor, tmo_flag);
        stage_end(h, st, a, kStageQbOrth);
    }
    if (e == cudaSuccess) {
        a = stage_begin(h, st);
        e = re::launch_qb_product(P.A, Q, ldq, k, B, ldb, h->qbws.p, tensor, static_cast<int*>(h->status.p) + 1, st,
                                  &nl);
        stage_end(h, st, a, kStageQbProduct);
    }
    h->stats.launches += nl;
    int hf = 0, tmo = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hf, floored, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&tmo, static_cast<int*>(h->status.p) + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "thin QR and B = Q^T A");
    if (tmo) return fail(RE_ERR_TIMEOUT, "a bounded device wait expired");
    if (hf) out->flags |= RE_QB_DEFLATED;
    resolve_timings(h);
    return RE_OK;
}

int check_opts(const re_opts* o) {
    if (o->s0 < 8 || o->s0 % 8 != 0) return fail(RE_ERR_ARG, "s0 must be a positive multiple of 8");
    if (o->s_max < o->s0) return fail(RE_ERR_ARG, "s_max < s0");
    if (o->s_max > 512) return fail(RE_ERR_ARG, "s_max above 512");
    if (o->precision != RE_PREC_FP32 && o->precision != RE_PREC_BF16X3 && o->precision != RE_PREC_EXACT)
        return fail(RE_ERR_ARG, "unknown precision");
    if (o->y_kind < -1 || o->y_kind == RE_HRTT || o->y_kind > RE_SRCT) return fail(RE_ERR_ARG, "unknown y_kind");
    if (o->learned != 0 && o->learned != 1) return fail(RE_ERR_ARG, "learned must be 0 or 1");
    if (o->test_drop_load != 0 && o->test_drop_load != 1) return fail(RE_ERR_ARG, "test_drop_load must be 0 or 1");
    if (o->sigma_est != RE_SIGMA_SVD && o->sigma_est != RE_SIGMA_QRDIAG) return fail(RE_ERR_ARG, "unknown sigma_est");
    if (o->batch_first_width < 0 || o->batch_first_width % 8 != 0)
        return fail(RE_ERR_ARG, "batch_first_width must be 0 or a positive multiple of 8");
    if (o->first_width < 0 || o->first_width % 8 != 0)
        return fail(RE_ERR_ARG, "first_width must be 0 or a positive multiple of 8");
    if (o->first_width > 0 && o->learned) return fail(RE_ERR_ARG, "first_width and learned exclude each other");
    if (o->sigma_est == RE_SIGMA_QRDIAG && o->precision == RE_PREC_EXACT)
        return fail(RE_ERR_UNSUPPORTED, "QR-diagonal estimates are FP32: not with the exact-product precision mode");
    return RE_OK;
}

}  // namespace

extern "C" {

int re_version(void) { return 100; }

const char* re_last_error(void) { return g_last_error.c_str(); }

void re_opts_default(re_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->s0 = 8;
    o->s_max = 512;
    o->precision = RE_PREC_FP32;
    o->y_kind = -1;
    o->norm_a = 0.0;
    o->learned = 0;
}

int re_create(re_handle* out, int device, const re_opts* opts) {
    if (!out) return fail(RE_ERR_ARG, "out is NULL");
    *out = nullptr;
    re_opts o;
    re_opts_default(&o);
    if (opts) o = *opts;
    if (int r = check_opts(&o)) return r;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(RE_ERR_ARG, "no such device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    re_handle h = new re_handle_();
    h->device = device;
    h->opts = o;
    cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, device);
    e = cudaMallocHost(reinterpret_cast<void**>(&h->h_ro), sizeof(re::DevReadoff));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&h->h_sigma), 1024 * sizeof(double));
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "pinned host buffers");
    }
    *out = h;
    return RE_OK;
}

int re_destroy(re_handle h) {
    if (!h) return RE_OK;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&h->x, &h->xt, &h->ax, &h->part, &h->core, &h->sigma, &h->sigma_scaled,
                      &h->svdws, &h->acopy, &h->dx, &h->px, &h->dy, &h->py, &h->ro, &h->status, &h->ht, &h->fz,
                      &h->qbws, &h->qbsel, &h->ctab, &h->ctabx,
                      &h->ex_rexp, &h->ex_xd, &h->ex_tr, &h->ex_hi, &h->ex_lo, &h->ex_cexp, &h->ex_yd, &h->ex_tc,
                      &h->ex_svd,
                      &h->mlp_P, &h->mlp_M, &h->mlp_V, &h->mlp_G, &h->mlp_X, &h->mlp_y,
                      &h->mlp_logits, &h->mlp_keep, &h->mlp_cls, &h->mlp_feat, &h->mlp_loss};
    for (DevBuf* b : bufs) release(*b);
    re::batched_destroy(h->batched);
    resolve_timings(h);
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : h->chunk_events) cudaEventDestroy(e);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->h_ro) cudaFreeHost(h->h_ro);
    if (h->h_sigma) cudaFreeHost(h->h_sigma);
    delete h;
    return RE_OK;
}

int re_stats_enable(re_handle h, int timing_on) {
    if (!h) return fail(RE_ERR_ARG, "NULL handle");
    h->timing = timing_on != 0;
    return RE_OK;
}

int re_stats_reset(re_handle h) {
    if (!h) return fail(RE_ERR_ARG, "NULL handle");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    resolve_timings(h);
    std::memset(&h->stats, 0, sizeof(h->stats));
    return RE_OK;
}

int re_stats_get(re_handle h, re_stats* out) {
    if (!h || !out) return fail(RE_ERR_ARG, "NULL argument");
    *out = h->stats;
    return RE_OK;
}

int re_set_opts(re_handle h, const re_opts* opts) {
    if (!h || !opts) return fail(RE_ERR_ARG, "NULL argument");
    if (int r = check_opts(opts)) return r;
    h->opts = *opts;
    return RE_OK;
}

int re_rank_estimate(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld,
                     double eps, int sketch_kind, uint64_t seed, double* sigma_out, int sigma_cap,
                     re_result* out, void* stream) {
    if (!h || !out) return fail(RE_ERR_ARG, "NULL handle or result");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    if (sigma_cap > 0 && !sigma_out) return fail(RE_ERR_ARG, "sigma_out is NULL");
    cudaSetDevice(h->device);
    const int ykind = left_kind(h, sketch_kind);
    Plan P;
    if (int r = make_plan(A, dtype, m, n, ld, sketch_kind, ykind, h->opts.s_max, &P)) return r;
    return run_estimate(h, P, eps, seed, sigma_out, sigma_cap, out,
                        static_cast<cudaStream_t>(stream));
}

int re_rank_estimate_host(re_handle h, const void* A_host, int dtype, int64_t m, int64_t n,
                          int64_t ld, double eps, int sketch_kind, uint64_t seed, double* sigma_out,
                          int sigma_cap, re_result* out, void* stream) {
    if (!h || !out || !A_host) return fail(RE_ERR_ARG, "NULL argument");
    if (m <= 0 || n <= 0 || ld < n) return fail(RE_ERR_ARG, "bad shape");
    if (dtype != RE_F32 && dtype != RE_F64) return fail(RE_ERR_ARG, "bad dtype");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    if (sigma_cap > 0 && !sigma_out) return fail(RE_ERR_ARG, "sigma_out is NULL");
    cudaSetDevice(h->device);
    const size_t es = dtype == RE_F32 ? 4 : 8;
    if (int r = ensure(h->acopy, es * (size_t)m * n)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const re_opts& o = h->opts;
    const bool pipe = dtype == RE_F32 && m >= n && sketch_kind == RE_GAUSSIAN && !o.learned &&
                      (o.precision == RE_PREC_BF16X3 || o.precision == RE_PREC_FP32);
    if (!pipe) {
        // contiguous rows: one linear copy (the 2-D form would be issued row by row)
        cudaError_t e = ld == n ? cudaMemcpyAsync(h->acopy.p, A_host, es * (size_t)m * n, cudaMemcpyHostToDevice, st)
                                : cudaMemcpy2DAsync(h->acopy.p, es * n, A_host, es * ld, es * n, m,
                                                    cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "host to device copy of A");
        return re_rank_estimate(h, h->acopy.p, dtype, m, n, n, eps, sketch_kind, seed, sigma_out,
                                sigma_cap, out, stream);
    }
    Plan P;
    if (int r = make_plan(h->acopy.p, dtype, m, n, n, sketch_kind, left_kind(h, sketch_kind), o.s_max, &P)) return r;
    if (o.s0 > P.cap) return fail(RE_ERR_ARG, "initial sketch width exceeds the admissible width");
    int smax = o.s0;
    while (smax * 2 <= P.cap) smax *= 2;
    int w1 = o.s0;
    while (w1 * 2 <= std::min(o.first_width, smax)) w1 *= 2;
    if (int r = ensure(h->ax, sizeof(float) * (size_t)m * smax)) return r;
    float* AX = static_cast<float*>(h->ax.p);
    // chunks of whole 128-row tiles; the copy stream starts after the caller's
    // earlier work on `stream` (which may still read the device copy of A)
    constexpr int kChunks = 8;
    const int64_t rows_per = std::max<int64_t>(128, ((m + kChunks - 1) / kChunks + 127) / 128 * 128);
    const int nch = (int)((m + rows_per - 1) / rows_per);
    cudaError_t e = cudaSuccess;
    if (!h->copy_stream) e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
    while (e == cudaSuccess && (int)h->chunk_events.size() < nch + 1) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) h->chunk_events.push_back(ev);
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy stream and events");
    e = cudaEventRecord(h->chunk_events[nch], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_stream, h->chunk_events[nch], 0);
    char* dst = static_cast<char*>(h->acopy.p);
    const char* src = static_cast<const char*>(A_host);
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        const int64_t r0 = (int64_t)c * rows_per, rc = std::min(rows_per, m - r0);
        e = ld == n ? cudaMemcpyAsync(dst + es * (size_t)r0 * n, src + es * (size_t)r0 * ld, es * (size_t)rc * n,
                                      cudaMemcpyHostToDevice, h->copy_stream)
                    : cudaMemcpy2DAsync(dst + es * (size_t)r0 * n, es * n, src + es * (size_t)r0 * ld, es * ld,
                                        es * n, rc, cudaMemcpyHostToDevice, h->copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(h->chunk_events[c], h->copy_stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "chunked host to device copy of A");
    // first pass chunk by chunk as the rows land (the rows of AX are independent)
    for (int c = 0; c < nch; ++c) {
        const int64_t r0 = (int64_t)c * rows_per, rc = std::min(rows_per, m - r0);
        e = cudaStreamWaitEvent(st, h->chunk_events[c], 0);
        if (e != cudaSuccess) return cuda_fail(e, "wait for a copied chunk");
        Plan Pc = P;
        Pc.A.ptr = dst + es * (size_t)r0 * n;
        Pc.A.rows = rc;
        if (int r = right_columns(h, Pc, seed, 0, w1, AX + (size_t)r0 * smax, smax, st)) return r;
    }
    return run_estimate(h, P, eps, seed, sigma_out, sigma_cap, out, st, w1);
}

int re_rank_estimate_qb(re_handle h, const float* A, int64_t m, int64_t n, int64_t ld, double eps, int p,
                        uint64_t seed, float* Q, int64_t ldq, float* B, int64_t ldb, int k_cap, re_qb_result* out,
                        void* stream) {
    if (!h || !A || !Q || !B || !out) return fail(RE_ERR_ARG, "NULL argument");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    if (p < 2) return fail(RE_ERR_ARG, "p must be at least 2");
    if (k_cap < 1) return fail(RE_ERR_ARG, "k_cap must be positive");
    cudaSetDevice(h->device);
    Plan P;
    if (int r = make_plan(A, RE_F32, m, n, ld, RE_GAUSSIAN, left_kind(h, RE_GAUSSIAN), h->opts.s_max, &P)) return r;
    if (ldb < P.A.cols) return fail(RE_ERR_ARG, "ldb < min(m, n)");
    return run_qb(h, P, eps, p, seed, Q, ldq, B, ldb, k_cap, out, static_cast<cudaStream_t>(stream));
}

int re_sketch_apply(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld,
                    int col0, int s, int sketch_kind, uint64_t seed, float* AX, int64_t ld_ax,
                    double* core, int64_t ld_core, void* stream) {
    if (!h || !AX) return fail(RE_ERR_ARG, "NULL argument");
    if (col0 < 0 || col0 % 8 != 0 || s <= 0 || s % 8 != 0)
        return fail(RE_ERR_ARG, "col0 and s must be multiples of 8, s > 0");
    if (ld_ax < col0 + s) return fail(RE_ERR_ARG, "ld_ax < col0 + s");
    if (core && ld_core < col0 + s) return fail(RE_ERR_ARG, "ld_core < col0 + s");
    cudaSetDevice(h->device);
    const int ykind = left_kind(h, sketch_kind);
    Plan P;
    if (int r = make_plan(A, dtype, m, n, ld, sketch_kind, ykind, 1 << 30, &P)) return r;
    if ((sketch_kind == RE_SRHT || hashed(sketch_kind)) && col0 + s > P.n_pad)
        return fail(RE_ERR_ARG, "SRHT/HRTT/HRCT width exceeds the padded dimension");
    if (hashed(sketch_kind) && col0 != 0)
        return fail(RE_ERR_ARG, "HRTT/HRCT columns depend on the width: col0 must be 0");
    if (core && ykind == RE_SRHT && 2 * (int64_t)(col0 + s) > P.m_pad)
        return fail(RE_ERR_ARG, "SRHT left width exceeds the padded dimension");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (exact_mode(h, P))
        return fail(RE_ERR_UNSUPPORTED, "the exact-product precision mode writes FP64 A X: use re_sketch_apply_exact");
    if (int r = right_columns(h, P, seed, col0, s, AX, ld_ax, st)) return r;
    if (core) {
        if (int r = left_blocks(h, P, seed, col0, col0 + s, AX, ld_ax, core, ld_core, st, 0)) return r;
    }
    return RE_OK;
}

int re_sketch_apply_exact(re_handle h, const float* A, int64_t m, int64_t n, int64_t ld, int col0, int s,
                          uint64_t seed, double* AX, int64_t ld_ax, double* core, int64_t ld_core, void* stream) {
    if (!h || !AX) return fail(RE_ERR_ARG, "NULL argument");
    if (col0 < 0 || col0 % 8 != 0 || s <= 0 || s % 8 != 0)
        return fail(RE_ERR_ARG, "col0 and s must be multiples of 8, s > 0");
    if (col0 + s > 512) return fail(RE_ERR_ARG, "col0 + s above 512");
    if (ld_ax < col0 + s) return fail(RE_ERR_ARG, "ld_ax < col0 + s");
    if (core && ld_core < col0 + s) return fail(RE_ERR_ARG, "ld_core < col0 + s");
    cudaSetDevice(h->device);
    Plan P;
    if (int r = make_plan(A, RE_F32, m, n, ld, RE_GAUSSIAN, RE_GAUSSIAN, 1 << 30, &P)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int c1 = col0 + s;
    if (int r = exact_prepare(h, P, c1, st)) return r;
    if (int r = ensure(h->status, 64)) return r;
    cudaError_t e = cudaMemsetAsync(h->status.p, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "clear status");
    if (int r = right_columns_exact(h, P, seed, col0, s, AX + col0, ld_ax, st)) return r;
    if (core) {
        // the caller's earlier columns of A X become the pair planes of the left sketch
        if (col0 > 0) {
            int* cexp = static_cast<int*>(h->ex_cexp.p);
            e = cudaMemsetAsync(cexp, 0x80, sizeof(int) * (size_t)col0, st);
            if (e == cudaSuccess)
                e = re::launch_f64_to_pairs(AX, ld_ax, P.A.rows, col0, static_cast<float*>(h->ex_hi.p),
                                            static_cast<float*>(h->ex_lo.p), h->ex_ldp, cexp, st);
            if (e != cudaSuccess) return cuda_fail(e, "earlier columns of A X");
            h->stats.launches += 2;
        }
        if (int r = left_blocks_exact(h, P, seed, col0, c1, core, ld_core, st, 0)) return r;
    }
    int tmo = 0;
    e = cudaMemcpyAsync(&tmo, static_cast<int*>(h->status.p) + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "exact sketch step");
    resolve_timings(h);
    if (tmo) return fail(RE_ERR_TIMEOUT, "a bounded device wait expired");
    return RE_OK;
}

int re_core_sigma(re_handle h, const double* core, int r2, int s, int64_t ld, double* sigma,
                  void* stream) {
    if (!h || !core || !sigma) return fail(RE_ERR_ARG, "NULL argument");
    if (s < 1 || s > 512 || r2 < s || r2 > 1024 || ld < s)
        return fail(RE_ERR_ARG, "need 1 <= s <= 512, s <= r2 <= 1024, ld >= s");
    cudaSetDevice(h->device);
    if (int r = ensure(h->svdws, re::svd_workspace_bytes(r2, s))) return r;
    if (int r = ensure(h->status, 64)) return r;
    cudaError_t e = re::launch_core_sigma(core, r2, s, ld, h->svdws.p, sigma,
                                          static_cast<int*>(h->status.p),
                                          static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "core singular values");
    return RE_OK;
}

int re_core_sigma_exact(re_handle h, const double* core, int r2, int s, int64_t ld, double* sigma, void* stream) {
    if (!h || !core || !sigma) return fail(RE_ERR_ARG, "NULL argument");
    if (s < 1 || s > 512 || r2 < s || r2 > 1024 || ld < s)
        return fail(RE_ERR_ARG, "need 1 <= s <= 512, s <= r2 <= 1024, ld >= s");
    cudaSetDevice(h->device);
    if (int r = ensure(h->svdws, re::svd_workspace_bytes(r2, s))) return r;
    if (int r = ensure(h->ex_svd, re::svd_precise_bytes(r2, s))) return r;
    if (int r = ensure(h->status, 64)) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = re::launch_core_sigma_precise(core, r2, s, ld, h->svdws.p, h->ex_svd.p, sigma,
                                                  static_cast<int*>(h->status.p), st);
    if (e != cudaSuccess) return cuda_fail(e, "core singular values (precise)");
    int stv = 0;
    e = cudaMemcpyAsync(&stv, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "core singular values (precise)");
    if (stv != RE_OK) return fail(stv, "non-finite values in the core");
    return RE_OK;
}

int re_embedding_x(re_handle h, int kind, uint64_t seed, int64_t n, int col0, int s, float* out,
                   void* stream) {
    if (!h || !out || n <= 0 || col0 < 0 || s <= 0) return fail(RE_ERR_ARG, "bad argument");
    if (kind == RE_GAUSSIAN && (col0 % 4 != 0)) return fail(RE_ERR_ARG, "col0 must be a multiple of 4");
    cudaSetDevice(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (kind == RE_GAUSSIAN) {
        e = re::launch_gauss_x(seed, n, col0, s, out, s, st);
    } else if (kind == RE_SRHT) {
        const int bits = re::pow2_bits(n);
        if (col0 + s > (int64_t(1) << bits)) return fail(RE_ERR_ARG, "SRHT width exceeds the padded dimension");
        if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)((int64_t(1) << bits) / 32 + 1))) return r;
        if (int r = ensure(h->px, sizeof(int) * (size_t)s)) return r;
        e = re::launch_sign_bits(seed, re::kStreamDX, n, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_perm(seed, re::kStreamPX, bits, col0, s, static_cast<int*>(h->px.p), st);
        if (e == cudaSuccess)
            e = re::launch_srtt_x_dense(n, s, static_cast<const uint32_t*>(h->dx.p),
                                        static_cast<const int*>(h->px.p), out, s, st);
    } else if (kind == RE_HRTT) {
        const int bits = re::pow2_bits(n);
        if (bits > 15) return fail(RE_ERR_UNSUPPORTED, "HRTT of more than 2^15 points");
        if (col0 != 0) return fail(RE_ERR_ARG, "HRTT columns depend on the width: col0 must be 0");
        if (s > (int64_t(1) << bits)) return fail(RE_ERR_ARG, "HRTT width exceeds the padded dimension");
        if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)((int64_t(1) << bits) / 32 + 1))) return r;
        if (int r = ensure(h->ht, sizeof(uint16_t) * (size_t)(int64_t(1) << bits))) return r;
        e = re::launch_sign_bits(seed, re::kStreamDX, n, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_hrtt_table(seed, bits, static_cast<uint16_t*>(h->ht.p), st);
        if (e == cudaSuccess)
            e = re::launch_hrtt_x_dense(n, s, bits, static_cast<const uint32_t*>(h->dx.p),
                                        static_cast<const uint16_t*>(h->ht.p), out, s, st);
    } else if (kind == RE_HRCT) {
        const int bits = re::pow2_bits(n);
        if (bits > 15) return fail(RE_ERR_UNSUPPORTED, "HRCT of more than 2^15 points");
        if (col0 != 0) return fail(RE_ERR_ARG, "HRCT columns depend on the width: col0 must be 0");
        if (s > (int64_t(1) << bits)) return fail(RE_ERR_ARG, "HRCT width exceeds the padded dimension");
        if (int r = ensure(h->dx, sizeof(uint32_t) * (size_t)((int64_t(1) << bits) / 32 + 1))) return r;
        if (int r = ensure(h->ht, sizeof(uint16_t) * (size_t)(int64_t(1) << bits))) return r;
        if (int r = ensure(h->ctabx, sizeof(float) * (size_t)((int64_t(1) << bits) + 1))) return r;
        e = re::launch_sign_bits(seed, re::kStreamDX, n, static_cast<uint32_t*>(h->dx.p), st);
        if (e == cudaSuccess) e = re::launch_hrtt_table(seed, bits, static_cast<uint16_t*>(h->ht.p), st);
        if (e == cudaSuccess) e = re::launch_cos_table(bits, static_cast<float*>(h->ctabx.p), st);
        if (e == cudaSuccess)
            e = re::launch_hrct_x(n, 0, s, 0, s, bits, static_cast<const uint32_t*>(h->dx.p),
                                  static_cast<const uint16_t*>(h->ht.p), static_cast<const float*>(h->ctabx.p), 0,
                                  out, nullptr, s, 0, st);
    } else {
        return fail(RE_ERR_ARG, "unknown kind");
    }
    if (e != cudaSuccess) return cuda_fail(e, "embedding X");
    return RE_OK;
}

int re_embedding_y(re_handle h, int kind, uint64_t seed, int64_t m, int row0, int r2, float* out,
                   void* stream) {
    if (!h || !out || m <= 0 || row0 < 0 || r2 <= 0) return fail(RE_ERR_ARG, "bad argument");
    if (kind == RE_GAUSSIAN && (row0 % 4 != 0)) return fail(RE_ERR_ARG, "row0 must be a multiple of 4");
    cudaSetDevice(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (kind == RE_GAUSSIAN) {
        e = re::launch_gauss_y(seed, m, row0, r2, out, m, st);
    } else if (kind == RE_SRHT) {
        const int bits = re::pow2_bits(m);
        if (row0 + r2 > (int64_t(1) << bits)) return fail(RE_ERR_ARG, "SRHT height exceeds the padded dimension");
        if (int r = ensure(h->dy, sizeof(uint32_t) * (size_t)((int64_t(1) << bits) / 32 + 1))) return r;
        if (int r = ensure(h->py, sizeof(int) * (size_t)r2)) return r;
        e = re::launch_sign_bits(seed, re::kStreamDY, m, static_cast<uint32_t*>(h->dy.p), st);
        if (e == cudaSuccess) e = re::launch_perm(seed, re::kStreamPY, bits, row0, r2, static_cast<int*>(h->py.p), st);
        if (e == cudaSuccess)
            e = re::launch_srtt_y_dense(m, r2, static_cast<const uint32_t*>(h->dy.p),
                                        static_cast<const int*>(h->py.p), out, m, st);
    } else {
        return fail(RE_ERR_ARG, "unknown kind");
    }
    if (e != cudaSuccess) return cuda_fail(e, "embedding Y");
    return RE_OK;
}

int re_rank_estimate_kernel_blocks(re_handle h, const re_kblock* blocks, int count, double eps, uint64_t seed,
                                   double* sigma_out, int sigma_cap, re_result* out, void* stream) {
    if (!h || (count > 0 && (!blocks || !out))) return fail(RE_ERR_ARG, "NULL argument");
    if (count < 0) return fail(RE_ERR_ARG, "count < 0");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    if (h->opts.precision != RE_PREC_BF16X3)
        return fail(RE_ERR_UNSUPPORTED, "matrix-free kernel blocks need the tensor-core sketch (RE_PREC_BF16X3)");
    if (h->opts.learned || (h->opts.y_kind >= 0 && h->opts.y_kind != RE_GAUSSIAN))
        return fail(RE_ERR_UNSUPPORTED, "matrix-free kernel blocks take the plain ladder with Gaussian embeddings");
    if (count == 0) return RE_OK;
    cudaSetDevice(h->device);
    return re::batched_estimate(&h->batched, h->opts, nullptr, blocks, count, eps, seed, sigma_out,
                                sigma_out ? sigma_cap : 0, out, static_cast<cudaStream_t>(stream), &h->stats.launches);
}

int re_rank_estimate_batched(re_handle h, const re_block* blocks, int count, int dtype, double eps,
                             int sketch_kind, uint64_t seed, double* sigma_out, int sigma_cap,
                             re_result* out, void* stream) {
    if (!h || (count > 0 && (!blocks || !out))) return fail(RE_ERR_ARG, "NULL argument");
    if (count < 0) return fail(RE_ERR_ARG, "count < 0");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    if (count == 0) return RE_OK;
    cudaSetDevice(h->device);
    const int ykind = left_kind(h, sketch_kind);
    if (dtype == RE_F32 && sketch_kind == RE_GAUSSIAN && ykind == RE_GAUSSIAN && !h->opts.learned) {
        // one graph launch over all blocks (level-synchronous batched kernels)
        return re::batched_estimate(&h->batched, h->opts, blocks, nullptr, count, eps, seed, sigma_out,
                                    sigma_out ? sigma_cap : 0, out, static_cast<cudaStream_t>(stream),
                                    &h->stats.launches);
    }
    // other element types / embeddings: one estimate per block
    for (int i = 0; i < count; ++i) {
        double* so = sigma_out ? sigma_out + (size_t)i * std::max(sigma_cap, 0) : nullptr;
        const int r = re_rank_estimate(h, blocks[i].ptr, dtype, blocks[i].m, blocks[i].n, blocks[i].ld,
                                       eps, sketch_kind, seed + (uint64_t)i, so,
                                       so ? sigma_cap : 0, &out[i], stream);
        if (r != RE_OK) {
            if (r == RE_ERR_CUDA || r == RE_ERR_NOMEM) return r;
            std::memset(&out[i], 0, sizeof(out[i]));
            out[i].status = r;
        }
    }
    return RE_OK;
}

}  // extern "C"

// ---- sketch-size proposal network --------------------------------------------
namespace {

int mlp_alloc(re_handle h) {
    const size_t P = sizeof(float) * re::kMlpParams;
    if (int r = ensure(h->mlp_P, P)) return r;
    if (int r = ensure(h->mlp_M, P)) return r;
    if (int r = ensure(h->mlp_V, P)) return r;
    if (int r = ensure(h->mlp_G, P)) return r;
    if (int r = ensure(h->mlp_loss, sizeof(float))) return r;
    return RE_OK;
}

int mlp_batch_buffers(re_handle h, int count) {
    if (int r = ensure(h->mlp_X, sizeof(float) * re::kMlpIn * (size_t)count)) return r;
    if (int r = ensure(h->mlp_y, sizeof(int) * (size_t)count)) return r;
    if (int r = ensure(h->mlp_logits, sizeof(float) * re::kMlpOut * (size_t)count)) return r;
    if (int r = ensure(h->mlp_keep, sizeof(float) * 2 * re::kMlpHidden * (size_t)count)) return r;
    if (int r = ensure(h->mlp_cls, sizeof(int) * (size_t)count)) return r;
    return RE_OK;
}

const char kMagic[8] = {'R', 'E', 'M', 'L', 'P', 'v', '1', 0};

}  // namespace

extern "C" {

int re_mlp_init(re_handle h, uint64_t seed) {
    if (!h) return fail(RE_ERR_ARG, "NULL handle");
    cudaSetDevice(h->device);
    if (int r = mlp_alloc(h)) return r;
    std::vector<float> p(re::kMlpParams);
    re::mlp_init_host(p.data(), seed);
    cudaError_t e = cudaMemcpy(h->mlp_P.p, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->mlp_M.p, 0, sizeof(float) * re::kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(h->mlp_V.p, 0, sizeof(float) * re::kMlpParams);
    if (e != cudaSuccess) return cuda_fail(e, "mlp init");
    h->mlp_step = 0;
    h->mlp_ready = true;
    return RE_OK;
}

int re_mlp_set_params(re_handle h, const float* params, int count) {
    if (!h || !params || count != re::kMlpParams) return fail(RE_ERR_ARG, "need RE_MLP_PARAMS parameters");
    cudaSetDevice(h->device);
    if (int r = mlp_alloc(h)) return r;
    cudaError_t e = cudaMemcpy(h->mlp_P.p, params, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mlp set params");
    h->mlp_ready = true;
    return RE_OK;
}

int re_mlp_get_params(re_handle h, float* params, int count) {
    if (!h || !params || count != re::kMlpParams) return fail(RE_ERR_ARG, "need RE_MLP_PARAMS parameters");
    if (!h->mlp_ready) return fail(RE_ERR_ARG, "no network");
    cudaSetDevice(h->device);
    cudaError_t e = cudaMemcpy(params, h->mlp_P.p, sizeof(float) * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp get params");
    return RE_OK;
}

int re_mlp_save(re_handle h, const char* path) {
    if (!h || !path) return fail(RE_ERR_ARG, "NULL argument");
    if (!h->mlp_ready) return fail(RE_ERR_ARG, "no network");
    cudaSetDevice(h->device);
    std::vector<float> buf(3 * (size_t)re::kMlpParams);
    cudaError_t e = cudaMemcpy(buf.data(), h->mlp_P.p, sizeof(float) * re::kMlpParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + re::kMlpParams, h->mlp_M.p, sizeof(float) * re::kMlpParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(buf.data() + 2 * re::kMlpParams, h->mlp_V.p, sizeof(float) * re::kMlpParams, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp save copy");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(RE_ERR_ARG, "cannot open file for writing");
    const int32_t hdr[2] = {re::kMlpParams, h->mlp_step};
    bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(RE_ERR_ARG, "write failed");
    return RE_OK;
}

int re_mlp_load(re_handle h, const char* path) {
    if (!h || !path) return fail(RE_ERR_ARG, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(RE_ERR_ARG, "cannot open file");
    char magic[8];
    int32_t hdr[2];
    std::vector<float> buf(3 * (size_t)re::kMlpParams);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == re::kMlpParams &&
              std::fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(RE_ERR_ARG, "not a proposal-network file of this version");
    cudaSetDevice(h->device);
    if (int r = mlp_alloc(h)) return r;
    cudaError_t e = cudaMemcpy(h->mlp_P.p, buf.data(), sizeof(float) * re::kMlpParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->mlp_M.p, buf.data() + re::kMlpParams, sizeof(float) * re::kMlpParams, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->mlp_V.p, buf.data() + 2 * re::kMlpParams, sizeof(float) * re::kMlpParams, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "mlp load copy");
    h->mlp_step = hdr[1];
    h->mlp_ready = true;
    return RE_OK;
}

int re_mlp_predict(re_handle h, const float* X, int count, int* classes, float* logits) {
    if (!h || (count > 0 && (!X || !classes))) return fail(RE_ERR_ARG, "NULL argument");
    if (!h->mlp_ready) return fail(RE_ERR_ARG, "no network");
    if (count <= 0) return RE_OK;
    cudaSetDevice(h->device);
    if (int r = mlp_batch_buffers(h, count)) return r;
    cudaError_t e = cudaMemcpy(h->mlp_X.p, X, sizeof(float) * re::kMlpIn * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = re::mlp_forward(static_cast<float*>(h->mlp_P.p), static_cast<float*>(h->mlp_X.p), count,
                            static_cast<float*>(h->mlp_logits.p), nullptr, nullptr);
    if (e == cudaSuccess) e = re::mlp_argmax(static_cast<float*>(h->mlp_logits.p), count, static_cast<int*>(h->mlp_cls.p), nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(classes, h->mlp_cls.p, sizeof(int) * count, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && logits)
        e = cudaMemcpy(logits, h->mlp_logits.p, sizeof(float) * re::kMlpOut * count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp predict");
    return RE_OK;
}

int re_mlp_grad(re_handle h, const float* X, const int* y, int count, float* grad, float* loss) {
    if (!h || !X || !y || !grad || count <= 0) return fail(RE_ERR_ARG, "bad argument");
    if (!h->mlp_ready) return fail(RE_ERR_ARG, "no network");
    for (int i = 0; i < count; ++i)
        if (y[i] < 0 || y[i] >= re::kMlpOut) return fail(RE_ERR_ARG, "label out of range");
    cudaSetDevice(h->device);
    if (int r = mlp_batch_buffers(h, count)) return r;
    float* G = static_cast<float*>(h->mlp_G.p);
    cudaError_t e = cudaMemcpy(h->mlp_X.p, X, sizeof(float) * re::kMlpIn * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->mlp_y.p, y, sizeof(int) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(G, 0, sizeof(float) * re::kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(h->mlp_loss.p, 0, sizeof(float));
    if (e == cudaSuccess)
        e = re::mlp_forward(static_cast<float*>(h->mlp_P.p), static_cast<float*>(h->mlp_X.p), count,
                            static_cast<float*>(h->mlp_logits.p), static_cast<float*>(h->mlp_keep.p), nullptr);
    if (e == cudaSuccess)
        e = re::mlp_backward(static_cast<float*>(h->mlp_P.p), static_cast<float*>(h->mlp_X.p),
                             static_cast<int*>(h->mlp_y.p), count, static_cast<float*>(h->mlp_logits.p),
                             static_cast<float*>(h->mlp_keep.p), G, static_cast<float*>(h->mlp_loss.p), nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(grad, G, sizeof(float) * re::kMlpParams, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && loss) e = cudaMemcpy(loss, h->mlp_loss.p, sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "mlp grad");
    return RE_OK;
}

int re_mlp_train(re_handle h, const float* X, const int* y, int count, int epochs, int batch, float lr,
                 float weight_decay, uint64_t seed, float* epoch_loss) {
    if (!h || !X || !y || count <= 0 || epochs <= 0 || batch <= 0 || !(lr > 0.f))
        return fail(RE_ERR_ARG, "bad argument");
    if (!h->mlp_ready) return fail(RE_ERR_ARG, "no network (re_mlp_init or re_mlp_load first)");
    for (int i = 0; i < count; ++i)
        if (y[i] < 0 || y[i] >= re::kMlpOut) return fail(RE_ERR_ARG, "label out of range");
    cudaSetDevice(h->device);
    const int B = std::min(batch, count);
    if (int r = mlp_batch_buffers(h, B)) return r;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::vector<float> xb((size_t)B * re::kMlpIn);
    std::vector<int> yb(B);
    float* G = static_cast<float*>(h->mlp_G.p);
    float* P = static_cast<float*>(h->mlp_P.p);
    uint64_t rng = seed * 6364136223846793005ull + 1442695040888963407ull;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int i = count - 1; i > 0; --i) {           // Fisher-Yates with a 64-bit LCG
            rng = rng * 6364136223846793005ull + 1442695040888963407ull;
            const int j = (int)((rng >> 33) % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        double ep_loss = 0.0;
        int nb = 0;
        cudaError_t e = cudaMemset(h->mlp_loss.p, 0, sizeof(float));
        for (int b0 = 0; b0 + B <= count && e == cudaSuccess; b0 += B, ++nb) {
            for (int k = 0; k < B; ++k) {
                std::memcpy(&xb[(size_t)k * re::kMlpIn], X + (size_t)order[b0 + k] * re::kMlpIn, sizeof(float) * re::kMlpIn);
                yb[k] = y[order[b0 + k]];
            }
            e = cudaMemcpy(h->mlp_X.p, xb.data(), sizeof(float) * xb.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(h->mlp_y.p, yb.data(), sizeof(int) * B, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemset(G, 0, sizeof(float) * re::kMlpParams);
            if (e == cudaSuccess)
                e = re::mlp_forward(P, static_cast<float*>(h->mlp_X.p), B, static_cast<float*>(h->mlp_logits.p),
                                    static_cast<float*>(h->mlp_keep.p), nullptr);
            if (e == cudaSuccess)
                e = re::mlp_backward(P, static_cast<float*>(h->mlp_X.p), static_cast<int*>(h->mlp_y.p), B,
                                     static_cast<float*>(h->mlp_logits.p), static_cast<float*>(h->mlp_keep.p), G,
                                     static_cast<float*>(h->mlp_loss.p), nullptr);
            if (e == cudaSuccess)
                e = re::mlp_adam(P, G, static_cast<float*>(h->mlp_M.p), static_cast<float*>(h->mlp_V.p), lr,
                                 ++h->mlp_step, weight_decay, nullptr);
        }
        float tot = 0.f;
        if (e == cudaSuccess) e = cudaMemcpy(&tot, h->mlp_loss.p, sizeof(float), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "mlp train");
        ep_loss = nb > 0 ? tot / nb : 0.0;
        if (epoch_loss) epoch_loss[ep] = (float)ep_loss;
    }
    return RE_OK;
}

int re_mlp_features(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld, double eps,
                    uint64_t seed, float* features) {
    if (!h || !features) return fail(RE_ERR_ARG, "NULL argument");
    if (!(eps > 0.0 && eps < 1.0)) return fail(RE_ERR_ARG, "eps must lie in (0, 1)");
    cudaSetDevice(h->device);
    const int ykind = RE_GAUSSIAN;
    Plan P;
    if (int r = make_plan(A, dtype, m, n, ld, RE_GAUSSIAN, ykind, 16, &P)) return r;
    if (P.cap < 16) return fail(RE_ERR_ARG, "matrix too small for the s = 16 first sketch");
    cudaStream_t st = nullptr;
    const int64_t M = P.A.rows;
    if (int r = ensure(h->ax, sizeof(float) * (size_t)M * 16)) return r;
    if (int r = ensure(h->core, sizeof(double) * 2 * 16 * 16)) return r;
    if (int r = ensure(h->sigma, sizeof(double) * 16)) return r;
    if (int r = ensure(h->sigma_scaled, sizeof(double) * 16)) return r;
    if (int r = ensure(h->ro, sizeof(re::DevReadoff))) return r;
    if (int r = ensure(h->status, 64)) return r;
    if (int r = ensure(h->mlp_feat, sizeof(float) * re::kMlpIn)) return r;
    cudaError_t e0 = cudaMemsetAsync(h->status.p, 0, 4 * sizeof(int), st);
    if (e0 != cudaSuccess) return cuda_fail(e0, "clear status");
    float* AX = static_cast<float*>(h->ax.p);
    if (int r = right_columns(h, P, seed, 0, 16, AX, 16, st)) return r;
    if (int r = left_blocks(h, P, seed, 0, 16, AX, 16, static_cast<double*>(h->core.p), 16, st, 0)) return r;
    re::DevReadoff ro;
    int r1 = 0;
    if (int r = check_width(h, P, 16, 16, eps, &ro, &r1, st)) return r;
    cudaError_t e = re::mlp_features(static_cast<const double*>(h->sigma_scaled.p), eps, P.A.rows, P.A.cols,
                                     static_cast<float*>(h->mlp_feat.p), st);
    if (e == cudaSuccess) e = cudaMemcpy(features, h->mlp_feat.p, sizeof(float) * re::kMlpIn, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "features");
    return RE_OK;
}

}  // extern "C"
