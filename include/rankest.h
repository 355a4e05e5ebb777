/*
 * rankest.h - C ABI of librankest.so, a GB300 (sm_103a) implementation of the
 * randomized numerical-rank estimator of Meier & Nakatsukasa, "Fast Randomized
 * Numerical Rank Estimation for Numerically Low-Rank Matrices".
 *
 * The estimator (Algorithm 1, Sec. 5) forms the two-sided sketch Y*A*X of an
 * m x n matrix A (m >= n, Notation in Sec. 1): the right sketch A*X with an
 * n x s embedding X (Gaussian, Sec. 3.4, or a subsampled randomized Hadamard
 * transform, Eq. (Theta) in Sec. 4), the left sketch Y*(A*X) with a 2s x m
 * embedding Y ("randomized approximate orthogonalization", Sec. 4), the
 * singular values of the small 2s x s core (step 7), and the read-off of the
 * eps-rank (Definition 1, Sec. 1.1) from the threshold eps*||A|| and the gap
 * sigma_i / sigma_{i+1} (step 8), growing s by doubling and appending until the
 * threshold is crossed (step 8; Sec. 5 on the choice of r1).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Return value: RE_OK (0) or a negative RE_ERR_* code.  On error nothing is
 *   written to caller outputs except where stated; re_last_error() gives a
 *   one-line message.
 * - A is row-major with leading dimension ld >= n (elements), FP32 or FP64
 *   (dtype RE_F32 / RE_F64).  FP64 input is rounded to FP32 as it is loaded.
 *   When m < n the estimate is taken on A^T (same eps-rank); results then carry
 *   RE_TRANSPOSED and "rows" below means the longer dimension.
 * - Device pointers are CUDA device memory of the handle's device; host
 *   pointers are ordinary (pageable or pinned) host memory.  The caller owns
 *   every buffer it passes; the library never frees them.
 * - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Work is stream-ordered; calls returning host values synchronise the stream.
 * - Sketch widths s are multiples of 8.  The ladder is s0, 2 s0, 4 s0, ...
 *   <= s_max; at width s the first r1(s) = max{r : round(1.1 r) <= s} sketched
 *   singular values are trusted (Algorithm 1 step 1 and Sec. 3.3's 10%
 *   oversampling), r2 = 2 s (step 4).
 * - Random embeddings are never passed in: they are drawn from a counter-based
 *   generator keyed by `seed` (Philox4x32-10, Box-Muller normals rounded to BF16,
 *   Feistel sampling for the SRHT), so a given seed always gives the same X and
 *   Y and larger widths append columns/rows to smaller ones.
 * - A handle is used by one host thread at a time.
 */
#ifndef RANKEST_H
#define RANKEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RE_OK 0
#define RE_ERR_ARG (-1)         /* invalid argument (null pointer, ld < n, eps not in (0,1), bad s) */
#define RE_ERR_CUDA (-2)        /* a CUDA runtime call failed */
#define RE_ERR_NONFINITE (-3)   /* A holds NaN or Inf (detected in the sketch) */
#define RE_ERR_TIMEOUT (-4)     /* a bounded device wait expired */
#define RE_ERR_NOMEM (-5)       /* device workspace allocation failed */
#define RE_ERR_UNSUPPORTED (-6) /* valid request this build does not handle */

/* element types of A */
#define RE_F32 0
#define RE_F64 1

/* embedding kinds (Sec. 3.4) */
#define RE_GAUSSIAN 0 /* iid N(0,1) entries, scaled by 1/sqrt(width) */
#define RE_SRHT 1     /* sqrt(N/r) S H D, H Sylvester Hadamard on the zero-padded dimension */
/* Hashed randomized Hadamard transform (Sec. 3.4, HRTT): X = D (H/sqrt(N)) C^T,
 * C a CountSketch (coordinate c in bucket pi^{-1}(c) mod s, random sign).  Right
 * embedding only; its columns depend on the width, so it is not appendable and
 * every doubling step sketches anew; the left embedding defaults to Gaussian. */
#define RE_HRTT 2
/* Subsampled randomized DCT (Eq. (Theta) with F the orthonormal DCT-II, eta = 2;
 * Sec. 4, the transform the paper's experiments use for Y): left embedding only
 * (opts.y_kind), sqrt(m_pad/r2) S F D on the zero-padded m_pad = 2^ceil(log2 m),
 * sampled frequencies pi_Y(q), signs D.  Its rows are generated on the fly from a
 * cosine table (m_pad + 1 FP32 values) inside the CUDA-core left sketch. */
#define RE_SRCT 3
/* Hashed randomized DCT (Sec. 3.4 with F the DCT-II in place of the Hadamard
 * transform; with the SRCT Y, the pair the paper's experiments use, Sec. 6): right
 * embedding only, X = D (F/sqrt(n_pad)) C^T with the HRTT's CountSketch C (buckets
 * {pi_X(k + t s)}, signs sigma_c) and D.  Every entry of X is an FP32 compensated
 * sum of its bucket's scaled cosines, generated densely (n x s) each pass; under
 * RE_PREC_BF16X3 the FP32 X enters the tensor cores as its three exact BF16 terms
 * (six products, 128 columns per launch), under RE_PREC_FP32 the CUDA-core sketch.
 * Like the HRTT it is not appendable (every doubling step sketches anew), its
 * width is at most n_pad <= 2^15, and the left embedding defaults to Gaussian. */
#define RE_HRCT 4

/* arithmetic of the Gaussian right sketch */
#define RE_PREC_FP32 0   /* FP32 FMA on CUDA cores */
#define RE_PREC_BF16X3 1 /* A split into three BF16 terms, tensor cores (tcgen05), FP32 accumulation */
/* Exact products and exact sums on the tensor cores: A (and A X for the left
 * sketch) cut into five 8-bit digits per entry relative to a power-of-two bound of
 * its row, the normals of X and Y into two (they are 16-bit fixed point), the
 * digit products summed exactly in FP32 accumulators over segments and in int64
 * across them; A X and Y A X are then exact up to one rounding at 2^-40 of their
 * rows' scale, and the core's singular values come from a preconditioned FP32
 * Jacobi (W = core V1 formed in FP64 from the FP32 right singular vectors V1, its
 * graded columns taken with a purely relative rotation test).  Resolves sketched
 * values down to about 1e-11 sigma_1 (Algorithm 1 at eps = 1e-8 on the
 * ten-decade spectra of Sec. 6).  Gaussian X and Y, FP32 A with m >= n, a
 * 16-byte aligned base and row pitch (ld a multiple of 4) and min(m, n) <= 2^20;
 * other inputs give RE_ERR_UNSUPPORTED. */
#define RE_PREC_EXACT 2

/* Step 7 (Algorithm 1): how the core's singular values are taken.
 * RE_SIGMA_SVD     singular values (QR + one-sided Jacobi).
 * RE_SIGMA_QRDIAG  the remark after Algorithm 1 (Sec. 5): |R_kk| of the core's
 *                  Householder QR, sorted descending, as estimates of the singular
 *                  values (a QR of a matrix whose right singular vectors are
 *                  randomised is rank-revealing with high probability); the
 *                  Jacobi sweeps are skipped.  Not with RE_PREC_EXACT. */
#define RE_SIGMA_SVD 0
#define RE_SIGMA_QRDIAG 1

/* result flags */
#define RE_CONVERGED 1u        /* some trusted sigma^_{i+1} <= eps ||A|| was found */
#define RE_LOWER_BOUND_ONLY 2u /* the ladder ended first: rank = r1(final s) is a lower bound (Sec. 5) */
#define RE_TRANSPOSED 4u       /* m < n: the estimate was taken on A^T */
#define RE_QB_DEFLATED 8u      /* Algorithm 3: a column of A X_k was numerically dependent on the
                                  earlier ones; the matching column of Q is zero */

typedef struct re_handle_* re_handle;

/* Options (all plain values).  re_opts_default() fills the defaults given here. */
typedef struct {
    int s0;          /* initial X width, multiple of 8 (default 8) */
    int s_max;       /* largest X width, <= 512 (default 512) */
    int precision;   /* RE_PREC_* for the Gaussian right sketch (default RE_PREC_FP32) */
    int y_kind;      /* left embedding kind: -1 = same as the right one (Gaussian for RE_HRTT
                        and RE_HRCT; default), RE_GAUSSIAN, RE_SRHT or RE_SRCT */
    double norm_a;   /* > 0: use as ||A|| in the threshold; otherwise sigma^_1 (step 8) */
    int learned;     /* 1: let the sketch-size proposal network pick the next width (default 0) */
    /* Test hook for the failure path (default 0; no counterpart in the paper): when
     * 1, CTA 0 of the tensor-core right sketch withholds its first A tile, so its
     * bounded waits expire (about 2 s); the call then returns RE_ERR_TIMEOUT and the
     * CUDA context stays usable.  Never set outside tests. */
    int test_drop_load;
    int sigma_est;   /* step 7: RE_SIGMA_SVD (default) or RE_SIGMA_QRDIAG */
    int batch_first_width; /* batched tensor-core ladder: width of its first pass; 0 (default) = autotuned */
    /* Single-matrix ladder (Gaussian X, FP32 or BF16x3): the first pass appends the
     * columns up to this width (a ladder width s0 2^j) in one read of A and the
     * read-off runs on the nested leading blocks of the core at s0, 2 s0, ... within
     * it: the plain ladder's rank, width and sigma with fewer passes (an HBM-bound
     * pass costs the same for 8 or 128 columns).  0 (default) = s0, the plain
     * ladder.  In re_rank_estimate_host the first pass runs under the
     * host-to-device copy, so a wide one (up to 256 columns) costs nothing there.
     * Not with learned = 1. */
    int first_width;
    int reserved[3];
} re_opts;

/* Outcome of one estimate.  sigma values go to a separate caller buffer. */
typedef struct {
    int rank;          /* eps-rank estimate r^ (or r1 with RE_LOWER_BOUND_ONLY) */
    int gap_index;     /* argmax_{1<=i<r1} sigma^_i / sigma^_{i+1}, smallest i on ties */
    double gap_ratio;  /* that ratio (+inf when sigma^_{i+1} = 0 < sigma^_i) */
    double tau;        /* the threshold eps * ||A|| used */
    int n_sigma;       /* r1(final_s): number of trusted sketched singular values */
    int final_s;       /* X width of the last step */
    int passes;        /* passes over A (sketch steps) */
    uint32_t flags;    /* RE_CONVERGED | RE_LOWER_BOUND_ONLY | RE_TRANSPOSED */
    int status;        /* per-estimate status (batched calls): RE_OK or RE_ERR_* */
    int svd_sweeps;    /* Jacobi sweeps used by the last small-core singular value step */
    int reserved[2];
} re_result;

/* One block of a batched estimate: a device matrix, row-major. */
typedef struct {
    const void* ptr;
    int64_t m, n, ld;
} re_block;

/* One matrix-free kernel block: K[i][j] = 1 / |x_i - y_j| for 3-D points x (m x 3)
 * and y (n x 3), device FP32, row-major (the structured blocks of Sec. 1 and
 * Sec. 3.4's remark that structure in A can make A X cheaper than a dense read). */
typedef struct {
    const float* x;
    const float* y;
    int64_t m, n;
} re_kblock;

/* Per-handle counters for measurement: kernel launches made by the library and,
 * when timing is enabled, CUDA-event time of each stage on the caller's stream.
 * right_bytes / right_flops are the algorithmic bytes (A read once, X read,
 * AX written) and flops of the right-sketch launches that were timed. */
typedef struct {
    int64_t launches;        /* kernels launched by this handle since the last reset */
    int64_t right_launches;  /* right-sketch kernel launches timed */
    double right_ms;         /* their summed device time */
    double right_bytes;      /* their algorithmic bytes */
    double right_flops;      /* their algorithmic flops */
    double left_ms;          /* left-sketch kernels (with the split-K reduction) */
    double svd_ms;           /* small-core singular values */
    double other_ms;         /* generator and read-off kernels */
    int64_t passes;          /* sketch passes over A */
    double qb_precondition_ms;   /* Algorithm 3: core Gram, R_s, W = A X_k R_s^{-1} */
    double qb_orthonormalise_ms; /* Algorithm 3: two Cholesky-QR passes on W */
    double qb_product_ms;        /* Algorithm 3: B = Q^T A */
    int64_t reserved[1];
} re_stats;

/* Library version as major*10000 + minor*100 + patch. */
int re_version(void);

/* Message for the last error on this host thread (static storage). */
const char* re_last_error(void);

/* Fill *opts with the defaults above. */
void re_opts_default(re_opts* opts);

/* Create a handle on CUDA device `device`.  opts may be NULL (defaults).  The
 * handle owns its device workspace, which grows on demand and is freed by
 * re_destroy. */
int re_create(re_handle* out, int device, const re_opts* opts);
int re_destroy(re_handle h);
int re_set_opts(re_handle h, const re_opts* opts);

/* Measurement counters (see re_stats).  Timing adds CUDA events around each
 * stage; it is off by default.  re_stats_get synchronises nothing: it reports
 * stages whose read-off step has completed. */
int re_stats_enable(re_handle h, int timing_on);
int re_stats_reset(re_handle h);
int re_stats_get(re_handle h, re_stats* out);

/*
 * Algorithm 1 with doubling (Sec. 5): estimate rank_eps(A).
 *   A          device pointer, m x n row-major, leading dimension ld.
 *   eps        relative tolerance in (0, 1) (Definition 1).
 *   sketch_kind RE_GAUSSIAN, RE_SRHT, RE_HRTT or RE_HRCT (right embedding; left
 *              per opts.y_kind, by default the same kind, Gaussian for the hashed
 *              RE_HRTT and RE_HRCT).  RE_SRHT / RE_HRTT / RE_HRCT take min(m, n) <=
 *              32768 (else RE_ERR_UNSUPPORTED); RE_HRTT or RE_HRCT with
 *              opts.learned is RE_ERR_UNSUPPORTED.
 *   seed       generator key for X and Y.
 *   sigma_out  host buffer of sigma_cap doubles, receives the first
 *              min(n_sigma, sigma_cap) scaled sketched singular values
 *              sigma_i(Y A X) (descending); may be NULL when sigma_cap = 0.
 *   out        host result.
 * Synchronises `stream` before returning.  A is only read.
 */
int re_rank_estimate(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld,
                     double eps, int sketch_kind, uint64_t seed,
                     double* sigma_out, int sigma_cap, re_result* out, void* stream);

/* As re_rank_estimate, but A is a HOST pointer: the call copies A to the
 * handle's device workspace (host->device inside the call) and reads back only
 * the result and sigma.  For FP32 A with m >= n, a Gaussian sketch and the
 * BF16x3 or FP32 precision (learned = 0), the copy runs in row chunks on a
 * stream of the handle while the first pass of the right sketch (s0 columns, or
 * opts.first_width) sketches each chunk on `stream` as it lands; the ladder then
 * continues on the device copy.  The result equals re_rank_estimate's up to the
 * rounding of A X (the tensor-core kernel's work split follows the row count). */
int re_rank_estimate_host(re_handle h, const void* A_host, int dtype, int64_t m, int64_t n,
                          int64_t ld, double eps, int sketch_kind, uint64_t seed,
                          double* sigma_out, int sigma_cap, re_result* out, void* stream);

/*
 * One appending sketch step (Algorithm 1 steps 2-6), for callers that reuse A*X
 * (randomized SVD / rangefinder, Sec. 5.1).  With k0 = col0:
 *   AX   device FP32, rows x ld_ax row-major (rows = max(m, n)); columns
 *        k0 .. k0+s-1 receive the UNSCALED right sketch A*G[:, k0:k0+s] (Gaussian G
 *        entries, or D H S^T entries +-1 for RE_SRHT).  Columns < k0 must hold
 *        earlier columns from the same seed when core is non-NULL.  RE_HRTT
 *        (col0 must be 0) writes the whole width-s sketch A D H C^T, RE_HRCT
 *        (col0 = 0) A D F^T C^T with F the DCT-II scaled to entries up to sqrt(2)
 *        (both unscaled: the caller applies 1/sqrt(N), N = 2^ceil(log2 min(m, n))).
 *   core optional device FP64, (2 (k0+s)) x ld_core row-major: on entry its
 *        leading 2 k0 x k0 block holds the previous unscaled core; on return the
 *        leading 2(k0+s) x (k0+s) block holds Y[0:2(k0+s)] * A * X[:, 0:k0+s].
 *        NULL skips the left sketch.
 * Scaling by 1/sqrt(width) is left to the caller.  col0 and s are multiples of 8.
 */
int re_sketch_apply(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld,
                    int col0, int s, int sketch_kind, uint64_t seed,
                    float* AX, int64_t ld_ax, double* core, int64_t ld_core, void* stream);

/*
 * re_sketch_apply for the exact-product precision mode (RE_PREC_EXACT, whatever
 * the handle's opts): Gaussian X and Y, FP32 A (m >= n, 16-byte aligned rows).
 *   AX   device FP64, rows x ld_ax row-major: columns col0 .. col0+s-1 receive the
 *        unscaled A*G[:, col0:col0+s], exact up to one rounding at 2^-40 of each
 *        row's power-of-two bound (then rounded to FP64).  When core is given,
 *        columns < col0 must hold the earlier columns (from this call's seed).
 *   core optional device FP64 as in re_sketch_apply (leading 2(col0+s) x (col0+s)
 *        block: Y[0:2(col0+s)] * A * X[:, 0:col0+s], exact to the same rounding).
 * col0 and s are multiples of 8, col0 + s <= 512.  Synchronises `stream`.
 */
int re_sketch_apply_exact(re_handle h, const float* A, int64_t m, int64_t n, int64_t ld, int col0, int s,
                          uint64_t seed, double* AX, int64_t ld_ax, double* core, int64_t ld_core, void* stream);

/*
 * Step 7 alone: the singular values of a device FP64 r2 x s matrix (row-major,
 * leading dimension ld), descending, written to the device FP64 array sigma
 * (s entries), unscaled.  1 <= s <= 512, s <= r2 <= 1024.  Computed by one-sided
 * Jacobi in FP32 (rotation round-off bounds the absolute error by about
 * 1e-5 * sigma_1).
 */
int re_core_sigma(re_handle h, const double* core, int r2, int s, int64_t ld,
                  double* sigma, void* stream);

/*
 * Step 7 alone with the precision mode's preconditioned singular values (same
 * arguments as re_core_sigma): FP32 QR + Jacobi of the core gives its right
 * singular vectors V1, W = core * V1 is formed in FP64, and the singular values
 * of W are taken by FP32 QR + Jacobi with a purely relative rotation test.  W's
 * columns are graded, so each value keeps its relative accuracy far below
 * u * sigma_1 (about 1e-12 * sigma_1 absolute).  Synchronises `stream`.
 */
int re_core_sigma_exact(re_handle h, const double* core, int r2, int s, int64_t ld,
                        double* sigma, void* stream);

/*
 * The embeddings themselves, for tests and for callers that want X or Y
 * explicitly (the estimator never materialises them this way):
 *   re_embedding_x: out (device FP32, n x s row-major) = columns col0.. of the
 *                   unscaled X (n = number of columns of the oriented A); for
 *                   RE_HRTT and RE_HRCT col0 = 0 and the s columns of the
 *                   width-s X.
 *   re_embedding_y: out (device FP32, r2 x m row-major) = rows row0.. of the
 *                   unscaled Y (m = number of rows of the oriented A).
 */
int re_embedding_x(re_handle h, int kind, uint64_t seed, int64_t n, int col0, int s,
                   float* out, void* stream);
int re_embedding_y(re_handle h, int kind, uint64_t seed, int64_t m, int row0, int r2,
                   float* out, void* stream);

/*
 * Batched Algorithm 1 over `count` independent blocks (e.g. the off-diagonal
 * blocks of a hierarchical matrix, Sec. 1).  blocks is a HOST array of device
 * matrices; out (host, count entries) receives one result each; sigma_out
 * (host, count x sigma_cap, may be NULL) the trusted sigma of each.  Every block
 * uses seed + block index.  Per-block argument errors are reported in
 * out[i].status; the call itself fails only on launch or allocation errors.
 * FP32 blocks with Gaussian embeddings run level-synchronously (all active
 * blocks advance one ladder width per level; widths up to min(s_max, 128)) as
 * ONE captured CUDA graph, replayed for repeated identical batches; other
 * cases run one estimate per block.  Synchronises `stream`.
 */
int re_rank_estimate_batched(re_handle h, const re_block* blocks, int count, int dtype,
                             double eps, int sketch_kind, uint64_t seed,
                             double* sigma_out, int sigma_cap, re_result* out, void* stream);

/* Result of re_rank_estimate_qb. */
typedef struct {
    int r;            /* target rank chosen by the Frobenius criterion (Algorithm 3 step 5) */
    int k;            /* columns of Q: r + p, or the last width when the criterion was not met */
    int final_s;      /* sketch width at which r was chosen */
    int passes;       /* reads of A by the sketch (B = Q^T A is one more) */
    uint32_t flags;   /* RE_CONVERGED: criterion met; RE_LOWER_BOUND_ONLY: the ladder ended
                         first; RE_TRANSPOSED: m < n, Q and B factor A^T;
                         RE_QB_DEFLATED: some columns of Q are zero (see below) */
    int status;       /* RE_OK, or RE_ERR_NONFINITE */
    double bound;     /* (1 + r/(p-1))^{1/2} (sum_{j>r} sigma^_j^2)^{1/2}: the estimated error */
    double norm_a;    /* ||A|| used by the criterion (sigma^_1 unless opts.norm_a) */
} re_qb_result;

/*
 * Algorithm 3 (Sec. 5.1): rank estimation combined with the randomized
 * rangefinder, for FP32 A (device, m x n row-major, ld).  The doubling ladder of
 * Algorithm 1 (Gaussian X; left embedding per opts.y_kind) runs until the
 * smallest r with (1 + r/(p-1))^{1/2} (sum_{j>r} sigma^_j^2)^{1/2} <= eps ||A||
 * (sigma^_j = sigma^_{r1} for r1 < j <= min(m, n), step 4) also has r + p <= s;
 * then Q (device FP32, max(m,n) x k, ldq >= k) gets orthonormal columns spanning
 * the first k = r + p columns of A X, and B = Q^T A (device FP32, k x min(m,n),
 * ldb >= min(m,n)), so A ~ Q B (A^T ~ Q B when m < n).  The thin QR uses the
 * core Y (A X_k) to precondition (Sec. 4's randomized approximate
 * orthogonalization) and two Cholesky-QR passes, all in the library's own
 * kernels (FP64 Gram of the core and FP64 blocked Cholesky factorizations and
 * triangular inverses; FP32 products on CUDA cores).  opts.precision selects
 * the ladder's sketch and B's product: RE_PREC_FP32 (FP32 SIMT sketch, B on
 * CUDA cores), RE_PREC_BF16X3 (tensor-core sketch; B = Q^T A on the tensor
 * cores with both factors split into three BF16 terms), RE_PREC_EXACT (the
 * exact-product sketch, which resolves the tail values step 5 sums, m >= n
 * only; B as for BF16X3).  A column of A X_k that
 * adds nothing resolvable to the span of the earlier ones (a Cholesky pivot below
 * 1e-24 of its squared norm for the core, 1e-12 in the FP32 passes: for example
 * columns at the FP32 noise floor when the ladder ends at s_max) is deflated:
 * its column of Q is zero and RE_QB_DEFLATED is set; the other columns stay
 * orthonormal and A ~ Q B holds as before.
 * p >= 2 (Halko et al. suggest 5 or 10).  If k exceeds k_cap, returns
 * RE_ERR_ARG with out->k set (call again with larger Q and B).  Synchronises
 * `stream`.
 */
int re_rank_estimate_qb(re_handle h, const float* A, int64_t m, int64_t n, int64_t ld, double eps, int p,
                        uint64_t seed, float* Q, int64_t ldq, float* B, int64_t ldb, int k_cap,
                        re_qb_result* out, void* stream);

/*
 * As re_rank_estimate_batched with Gaussian embeddings, for matrix-free kernel
 * blocks (HOST array of re_kblock): the tensor-core right sketch computes each
 * entry 1 / |x_i - y_j| in FP32 (differences, fused multiply-adds, the hardware
 * reciprocal square root, relative error below 2^-22) as it feeds the MMA, so
 * no block is ever stored.  Blocks with m < n are sketched as
 * K^T (the kernel is symmetric: the point sets swap roles), RE_TRANSPOSED set.
 * Needs opts.precision = RE_PREC_BF16X3 and neither opts.learned nor a non-Gaussian
 * opts.y_kind (else RE_ERR_UNSUPPORTED).  Coincident points give an infinite
 * entry and RE_ERR_NONFINITE in that block's status.  Synchronises `stream`.
 */
int re_rank_estimate_kernel_blocks(re_handle h, const re_kblock* blocks, int count, double eps,
                                   uint64_t seed, double* sigma_out, int sigma_cap, re_result* out,
                                   void* stream);

/*
 * Sketch-size proposal network (answers the question left open in the paper's
 * discussion, Sec. 7: choosing a new r1 from the information of a first run).
 * An 18 -> 128 -> 128 -> 12 ReLU network maps features of an s = 16 first sketch
 * (the 14 trusted log10(sigma^_i / (eps sigma^_1)), log10 rows, log10 cols,
 * log10(1/eps), and the log decay of the last seven trusted values) to a width
 * class c (width 8 * 2^c).  With opts.learned = 1, re_rank_estimate sketches to
 * s = 16, asks the network for s*, appends straight to s*, and checks the
 * read-off on the nested leading core blocks at s = 8, 16, 32, ..., s* in
 * order: the result equals the plain doubling ladder's whenever s* is at least
 * its final width, and doubling continues from s* otherwise.  Weights are used
 * in BF16 with FP32 accumulation (FP32 master copies, Adam).  All compute runs
 * in this library's kernels.  Parameter layout: W1 (128x18), b1, W2 (128x128),
 * b2, W3 (12x128), b3, row-major, RE_MLP_PARAMS floats.
 */
#define RE_MLP_IN 18
#define RE_MLP_OUT 12
#define RE_MLP_PARAMS 20492
int re_mlp_init(re_handle h, uint64_t seed);                        /* deterministic He-uniform init */
int re_mlp_set_params(re_handle h, const float* params, int count); /* host -> device */
int re_mlp_get_params(re_handle h, float* params, int count);       /* device -> host */
/* Versioned file: magic "REMLPv1", parameter count, Adam step, parameters and
 * both Adam moments (training resumes where it stopped). */
int re_mlp_save(re_handle h, const char* path);
int re_mlp_load(re_handle h, const char* path);
/* classes (host, count) = argmax of the logits of X (host, count x 18); logits may be NULL */
int re_mlp_predict(re_handle h, const float* X, int count, int* classes, float* logits);
/* gradient (host, RE_MLP_PARAMS) and value of the mean softmax cross-entropy at (X, y) */
int re_mlp_grad(re_handle h, const float* X, const int* y, int count, float* grad, float* loss);
/* Adam training on (X, y) (host arrays); epoch_loss (host, epochs entries) may be NULL */
int re_mlp_train(re_handle h, const float* X, const int* y, int count, int epochs, int batch, float lr,
                 float weight_decay, uint64_t seed, float* epoch_loss);
/* the 18 features of the s = 16 first sketch of a device matrix (Gaussian X, Y) */
int re_mlp_features(re_handle h, const void* A, int dtype, int64_t m, int64_t n, int64_t ld, double eps,
                    uint64_t seed, float* features);

/*
 * The Gaussian sketch step of re_sketch_apply without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory -- code running inside a CUDA stream capture (where
 * cudaMalloc would break the capture), applications whose device memory is owned
 * by their own pool or caching allocator, and real-time paths where an
 * allocation's latency or failure is not acceptable.  It needs no handle.
 *   Arguments and outputs are those of re_sketch_apply with sketch_kind =
 *   RE_GAUSSIAN and FP32 arithmetic (AX columns col0..col0+s-1 unscaled; the
 *   optional FP64 core appended in place).
 *   Scratch (the generated X columns and the left sketch's split-K partial sums)
 *   lives in one 16 MiB static device array that every GPU loading the library
 *   holds until exit; calls needing more (about min(m,n)*s + 2(col0+s)*s*splits
 *   floats > 4 Mi) return RE_ERR_ARG.
 *   The kernels run on the device that holds A (the current device is restored
 *   on return); AX and core must be device memory of that same device, else
 *   RE_ERR_ARG.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   All calls share the array: calls that overlap on the GPU race on it and must
 *   be serialised by the caller.  Nothing in it needs to start at zero.
 */
int re_sketch_apply_noalloc(const void* A, int dtype, int64_t m, int64_t n, int64_t ld, int col0,
                            int s, uint64_t seed, float* AX, int64_t ld_ax, double* core,
                            int64_t ld_core, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RANKEST_H */
