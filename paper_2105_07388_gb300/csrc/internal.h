// Internal interfaces between the translation units of librankest (not part of the C ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rankest.h"

namespace re {

// Records msg as the thread's last error (re_last_error) and returns code.
int set_last_error(int code, const char* msg);

// Oriented view of the caller's matrix: rows >= cols.  Element (r, c) of the
// oriented matrix sits at A[r*ld + c] (plain) or A[c*ld + r] (transposed).
struct MatView {
    const void* ptr;
    int dtype;      // RE_F32 / RE_F64
    int64_t rows;   // m' = max(m, n)
    int64_t cols;   // n' = min(m, n)
    int64_t ld;
    bool trans;
};

// One block of a batched estimate, as the batched kernels see it (device array).
struct BatchDesc {
    const float* A;     // FP32, oriented view as in MatView
    int64_t ld;
    int64_t rows, cols; // rows >= cols
    int trans;
    int smax;           // largest sketch width for this block
    int64_t ax_off;     // offset (floats) of this block's AX region (rows x ldax) in the AX pool
    int64_t x_off;      // offset (floats) of this block's X region (cols x xs) in the X pool
    uint64_t seed;
    int64_t xt_off;     // offset (BF16 elements) of this block's X^T region (nxt x kpad) in the X^T pool
    int64_t kpad;       // cols rounded up to a multiple of 64
    // matrix-free kernel block (A == nullptr): entry (r, c) of the oriented block
    // is 1 / |px[r] - py[c]| for 3-D points (FP32, 3 per point), trans == 0
    const float* px;
    const float* py;
    // tensor-core path: 1 (row-major block) or 2 (block stored transposed) when its
    // stored rows are fetched through four row-class tensor maps (stored rows c, c+4,
    // c+8, ... for c = 0..3); 0: asynchronous copies
    int tmaps;
};

// ---- embeddings (embed.cu) ----------------------------------------------------
// X columns [col0, col0+s) as FP32, row-major n x ldx.
cudaError_t launch_gauss_x(uint64_t seed, int64_t n, int col0, int s, float* X, int64_t ldx,
                           cudaStream_t st);
// X columns [col0, col0+s) as BF16 bits, column-major (s rows of n): Xt[j*ldt + k].
cudaError_t launch_gauss_xt_bf16(uint64_t seed, int64_t n, int64_t n_alloc, int col0, int s,
                                 uint16_t* Xt, int64_t ldt, cudaStream_t st);
// SRTT right embedding columns as BF16 bits: Xt[j][k] = d_k H[k][cols[j]] (+-1) for
// k < n, zero up to n_alloc; j < s; d from the sign bits (bit set = -1).
cudaError_t launch_srht_xt_bf16(int64_t n, int64_t n_alloc, const int* cols, const uint32_t* dbits, int s,
                                uint16_t* Xt, int64_t ldt, cudaStream_t st);
// Y rows [row0, row0+r2) as FP32, row-major r2 x ldy.
cudaError_t launch_gauss_y(uint64_t seed, int64_t m, int row0, int r2, float* Y, int64_t ldy,
                           cudaStream_t st);
// SRTT sign bits: bit j of words[j/32] set <=> d_j = -1, j < count (stream DX or DY).
cudaError_t launch_sign_bits(uint64_t seed, uint32_t stream, int64_t count, uint32_t* words,
                             cudaStream_t st);
// SRTT sampled indices pi(k0 .. k0+cnt-1) on `bits` bits (stream PX or PY).
cudaError_t launch_perm(uint64_t seed, uint32_t stream, int bits, int k0, int cnt, int* out,
                        cudaStream_t st);
// Dense SRTT X / Y entries (+-1) for re_embedding_x/y.
cudaError_t launch_srtt_x_dense(int64_t n, int s, const uint32_t* dbits, const int* cols, float* X,
                                int64_t ldx, cudaStream_t st);
cudaError_t launch_srtt_y_dense(int64_t m, int r2, const uint32_t* dbits, const int* rows, float* Y,
                                int64_t ldy, cudaStream_t st);
// HRTT hashing table of 2^bits entries (bits <= 15): entry q = pi_X(q) | (sigma < 0) << 15.
cudaError_t launch_hrtt_table(uint64_t seed, int bits, uint16_t* tbl, cudaStream_t st);
// Columns j0 .. j0+cnt-1 of the width-s hashed randomized DCT X (order 2^bits, the HRTT's
// buckets and signs from tbl, cosines from ctab = launch_cos_table(bits)): planes = 0
// writes FP32 X row-major (ldx, column j - j0); planes = 3 writes the three exact BF16
// terms of the FP32 values as X^T planes of plane_rows rows (row pitch ldx, zeros for
// n <= k < kpad).
cudaError_t launch_hrct_x(int64_t n, int64_t kpad, int s, int j0, int cnt, int bits, const uint32_t* dbits,
                          const uint16_t* tbl, const float* ctab, int planes, float* X, uint16_t* Xt, int64_t ldx,
                          int64_t plane_rows, cudaStream_t st);
// Rows j0 .. j0+cnt-1 of the width-s HRTT's X^T as BF16 bits (kpad per row, zero past
// n): Xt[j - j0][k] = d_k sum over bucket j of sigma_c H[k, c].  planes = 1: exact when
// every bucket holds at most 256 coordinates (2^bits <= 256 s); planes = 2: the
// entries' nearest BF16 in rows 0.., their remainders in rows plane_rows.. (exact
// for any bucket size up to 2^15).
cudaError_t launch_hrtt_xt_bf16(int64_t n, int64_t kpad, int s, int j0, int cnt, int bits, const uint32_t* dbits,
                                const uint16_t* tbl, uint16_t* Xt, int64_t ldt, cudaStream_t st, int planes = 1,
                                int64_t plane_rows = 0);
// Dense HRTT X (n x s, +-integer entries) for re_embedding_x.
cudaError_t launch_hrtt_x_dense(int64_t n, int s, int bits, const uint32_t* dbits, const uint16_t* tbl,
                                float* X, int64_t ldx, cudaStream_t st);

// ---- right sketch, FP32 SIMT (sketch_simt.cu) -------------------------------------
// C[:, 0:s] (row-major, ldc) = A_oriented * X[:, 0:s], X FP32 row-major n' x ldx.
cudaError_t launch_right_simt(const MatView& A, const float* X, int64_t ldx, int s, float* C,
                              int64_t ldc, cudaStream_t st);

// ---- left sketch (sketch_simt.cu) ---------------------------------------------
// core[row0+r][col0+c] (FP64, ld_core) = sum_i Y[row0+r][i] * AX[i][col0+c] for
// r < R, c < S, i < M, Y Gaussian.  `part` is FP32 scratch of part_cap floats.
// With a non-null err_flag (a device word that a bounded wait sets on expiry),
// blocks of aligned AX run on the tensor cores (left_tc.cu); otherwise, and when
// `part` is too small for that kernel's split count, on CUDA cores.
cudaError_t launch_left(uint64_t seed, const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0, int S,
                        float* part, size_t part_cap, double* core, int64_t ld_core, cudaStream_t st,
                        int* err_flag = nullptr);
size_t left_part_floats(int64_t M, int R, int S);
// Rows of the unscaled SRCT left embedding: Y[q][i] = sqrt(2) w_k cos(pi (2i+1) k / (2N)) d_i
// with k = krow[q], N = 2^nbits (w_0 = 1/sqrt(2), else 1), d_i from the sign bits (bit
// set = -1) and cos(pi j / (2N)) = ctab[j] for j in [0, N].
struct DctRows {
    const int* krow;
    const uint32_t* dbits;
    const float* ctab;
    int nbits;
};
// ctab[j] = cos(pi j / 2^(nbits+1)) for j in [0, 2^nbits] (FP32 from FP64 cospi).
cudaError_t launch_cos_table(int nbits, float* ctab, cudaStream_t st);
// core[row0+r][col0+c] (FP64) = sum_i Y[row0+r][i] AX[i][col0+c], Y the SRCT rows
// above (FP32 split-K partials in `part`, summed as for launch_left).  With a
// non-null err_flag, blocks of aligned AX run on the tensor cores (Y as three BF16
// terms; left_tc.cu) when `part` holds that kernel's partials, else on CUDA cores.
cudaError_t launch_left_dct(const DctRows& Y, const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0,
                            int S, float* part, size_t part_cap, double* core, int64_t ld_core, cudaStream_t st,
                            int* err_flag = nullptr);

// ---- left sketch with the SRTT Y by fast transforms (left_fwht.cu) ------------
// Z[i][c] = (H D AX)[i][c] for c in [c0, c1) and i < 2^mbits (Z row-major, ldz >= c1,
// 2^mbits rows; AX rows >= M are zero; dbits the DY signs).
cudaError_t launch_left_srtt_transform(const float* AX, int64_t ldax, int64_t M, int mbits, const uint32_t* dbits,
                                       int c0, int c1, float* Z, int64_t ldz, cudaStream_t st);
// core[row0+r][col0+c] = Z[perm[row0+r]][col0+c] for r < R, c < S (perm = pi_Y).
cudaError_t launch_left_srtt_sample(const float* Z, int64_t ldz, const int* perm, int row0, int R, int col0, int S,
                                    double* core, int64_t ld_core, cudaStream_t st);

// ---- left sketch on the tensor cores (left_tc.cu) -----------------------------
bool left_tc_supported(const float* AX, int64_t ldax, int64_t M, int row0, int R, int col0, int S);
size_t left_tc_part_floats(int64_t M, int R, int S, bool dct = false);
// FP32 split-K partials part[split][R][S] of the block; *splits_out = splits used.
// dct non-null: Y is the SRCT of those rows (three BF16 terms, six products).
cudaError_t launch_left_tc_partials(uint64_t seed, const float* AX, int64_t ldax, int64_t M, int row0, int R,
                                    int col0, int S, float* part, size_t part_cap, int* err_flag, int* splits_out,
                                    cudaStream_t st, const DctRows* dct = nullptr);

// Batched right sketch on the tensor cores (batched_tc.cu), BF16x3 as in
// right_tc_kernel: for every active block b and each of its 128-row tiles,
// AX_b[:, col0:col0+s] = A_b X_b with X_b^T BF16 in the X^T pool (nxt =
// tc_mma_n(s) rows of kpad, rows >= s zero).  act_prefix (count + 1 entries,
// from launch_compact_tiles) numbers the tiles of the active blocks; max_items
// bounds their number.  A is loaded with asynchronous copies of 16, 8 or 4
// bytes, so any row pitch works.
// It also writes tile_block[t] (max_items entries), the block of each active tile.
cudaError_t launch_compact_tiles(const BatchDesc* d, int count, const int* active, int64_t* act_prefix,
                                 int* tile_block, int64_t max_items, cudaStream_t st);
// tmaps: device array of 4 tensor maps per block (block b's at 4b .. 4b+3, used when
// d[b].tmaps is set; see encode_row_class_maps).
cudaError_t launch_right_tc_batched(const BatchDesc* d, int count, const int64_t* act_prefix, const int* tile_block,
                                    int64_t max_items, const uint16_t* XTpool, int s, float* AXpool, int64_t ldax,
                                    int col0, int* err_flag, const void* tmaps, cudaStream_t st);
// Bytes of one tensor map (CUtensorMap) of the row-class fetch.
size_t row_class_map_bytes();
// Encodes into out (4 maps) the row classes of an FP32 matrix stored row-major with
// srows x scols values, pitch ld: class c holds stored rows c, c+4, ... (pitch 16 ld
// bytes, always a multiple of 16) from the 16-byte boundary at or below its first
// row; boxes of box_x floats x box_y rows, zero fill past the stored columns and
// rows.  Returns false when a map cannot be encoded.
bool encode_row_class_maps(const float* A, int64_t ld, int64_t srows, int64_t scols, int box_x, int box_y,
                           void* out);
// X_b^T (BF16, nxt rows x kpad) of columns [col0, col0+s) for every active block.
cudaError_t launch_gauss_xt_batched(const BatchDesc* d, int count, const int* active, int col0, int s, int nxt,
                                    uint16_t* XTpool, cudaStream_t st);

// Batched right sketch: for every active block b and each of its BM-row tiles
// (tile_prefix[b] .. tile_prefix[b+1]-1 are b's work items), AX_b[:, col0:col0+s]
// = A_b X_b with X_b (cols x s, ld s) at Xpool + x_off.  BM is 64 or 128.
cudaError_t launch_right_simt_batched(const BatchDesc* d, int count, const int64_t* tile_prefix,
                                      int64_t items, const int* active, const float* Xpool, int s,
                                      float* AXpool, int64_t ldax, int col0, int bm, cudaStream_t st);

// ---- right sketch, SRHT (sketch_srht.cu) --------------------------------------
// C[:, 0:s] = A_oriented * D H S^T with sampled Hadamard columns cols[0..s).
cudaError_t launch_right_srht(const MatView& A, const uint32_t* dbits, const int* cols, int s,
                              float* C, int64_t ldc, cudaStream_t st, int* err = nullptr);
// C[:, 0:s] = A_oriented D H C^T (HRTT, unscaled): output k sums the transform
// coordinates of bucket k with their CountSketch signs, read from the table of
// launch_hrtt_table (pow2_bits(cols) bits).  Requires s <= 2^bits.  The table
// is reordered in place for the bulk kernel (entries stay in their buckets;
// only the order of each bucket's sum changes).
cudaError_t launch_right_hrtt(const MatView& A, const uint32_t* dbits, uint16_t* tbl, int s,
                              float* C, int64_t ldc, cudaStream_t st, int* err = nullptr);

// ---- right sketch, BF16x3 tensor cores (sketch_tc.cu) ------------------------------
bool tc_supported(const MatView& A);
// MMA N used for s output columns (>= 16, multiple of 16); X^T needs that many rows.
int tc_mma_n(int s);
// X^T holds xterms BF16 planes of tc_mma_n(s) rows each (plane t at row t * tc_mma_n(s)):
// 1 for BF16-exact X, 2 for X = hi + lo exactly, 3 for FP32 X (six products, error
// below 2^-24 of |A||X|); xterms > 1 takes at most 128 columns.
cudaError_t launch_right_tc(const MatView& A, const uint16_t* Xt, int64_t ldt, int s, float* C,
                            int64_t ldc, int* err_flag, cudaStream_t st, int* launches = nullptr,
                            int drop_first = 0, int xterms = 1);

// ---- exact-product sketches of the precision mode (sketch_ex.cu) --------------
// e[r] = smallest e with |A[r][k]| < 2^e (0 for a zero row); *status |= 1 for
// Inf/NaN, |= 2 for an entry of 2^126 or more.
cudaError_t launch_row_exponent(const float* A, int64_t ld, int64_t M, int64_t K, int* e, int* status,
                                cudaStream_t st);
// Two BF16 digit slices of Gaussian normals, K-major: slice t row r at D + (t slice_rows + r) ld,
// entries k < kpad (zero for k >= kvalid); row r is short index row0 + r of the
// embedding of `stream` (kStreamGX: X^T rows = X columns; kStreamGY: Y rows).
cudaError_t launch_normal_digits(uint64_t seed, uint32_t stream, int64_t kvalid, int64_t kpad, int row0, int rows,
                                 uint16_t* D, int64_t ld, int64_t slice_rows, cudaStream_t st);
// T[r][q] += exact sum_k P[r][k] Q[q][k] in units of 2^(e_r - 40) (int64, atomics; T
// must start at zero).  P FP32 row-major (ldp % 4 == 0, 16-byte aligned), or the pair
// P + P_lo; Q rows q_row0 .. q_row0 + N - 1 of the digit-slice array (ldq % 64 == 0,
// >= K rounded up to 64).  K <= 2^20.
cudaError_t launch_ex_sketch(const float* P, const float* P_lo, int64_t ldp, int64_t M, int64_t K, const int* rexp,
                             const uint16_t* Qd, int64_t ldq, int q_slice_rows, int q_row0, int N,
                             unsigned long long* T, int64_t ldt, int* err_flag, cudaStream_t st, int* launches);
// T (M x N, units 2^(rexp[r] - 40)) -> FP32 pair planes of the transpose (row c of the
// planes = column c, ld ldp; may be NULL), FP64 values V (row-major, ldv; may be NULL)
// and atomicMax of each column's exponent into cexp (set to INT_MIN-like before).
cudaError_t launch_ex_finalize(const long long* T, int64_t ldt, const int* rexp, int64_t M, int N, float* Phi,
                               float* Plo, int64_t ldp, double* V, int64_t ldv, int* cexp, cudaStream_t st);
// core[q_off + q][c_off + c] = T[c][q] 2^(cexp[c_off + c] - 40) for c < C, q < Q.
cudaError_t launch_ex_core_finalize(const long long* T, int64_t ldt, const int* cexp, int C, int Q, int c_off,
                                    int q_off, double* core, int64_t ld_core, cudaStream_t st);
// FP64 values (row-major M x N, ldv) -> FP32 pair planes of the transpose and column
// exponents (as launch_ex_finalize).
cudaError_t launch_f64_to_pairs(const double* V, int64_t ldv, int64_t M, int N, float* Phi, float* Plo, int64_t ldp,
                                int* cexp, cudaStream_t st);

// ---- small core singular values (core_svd.cu) ----------------------------------
size_t svd_workspace_bytes(int r2, int s);
// sigma (FP64, s entries, descending, unscaled) of core (FP64 row-major r2 x s, ld).
// status (device int): 0 ok, RE_ERR_NONFINITE if core has NaN/Inf.  ws: device
// scratch of svd_workspace_bytes(r2, s) bytes (16-byte aligned), used by the
// cluster path (cores that do not fit one CTA).
// With cert_r1 > 0 the one-CTA path first tries to certify that sigma_{cert_r1}
// exceeds cert_ratio * sigma_1 (then status[3] = 1 and sigma is left unwritten).
cudaError_t launch_core_sigma(const double* core, int r2, int s, int64_t ld, void* ws,
                              double* sigma, int* status, cudaStream_t st, int cert_r1 = 0,
                              float cert_ratio = 0.f);
// Step 7 by the QR diagonal (the remark after Algorithm 1): |R_kk| of the core's
// Householder QR (FP32), sorted descending, unscaled; no Jacobi.
cudaError_t launch_core_qrdiag(const double* core, int r2, int s, int64_t ld, void* ws, double* sigma, int* status,
                               cudaStream_t st);
// Precision-mode singular values (sigma descending, unscaled, status as above):
// the FP32 QR + Jacobi of the core gives right singular vectors V1; W = core V1
// (columns ordered by decreasing norm) is formed in FP64 and its singular values
// are taken by the same FP32 QR + Jacobi with a purely relative rotation test.
// W's columns are graded (about sigma_k u_k), and Householder QR and one-sided
// Jacobi are column-wise backward stable, so values far below u sigma_1 keep
// their relative accuracy; sigma(W) = sigma(core) up to the relative
// non-orthogonality of V1.  pws: svd_precise_bytes(r2, s) of device scratch.
size_t svd_precise_bytes(int r2, int s);
cudaError_t launch_core_sigma_precise(const double* core, int r2, int s, int64_t ld, void* ws, void* pws,
                                      double* sigma, int* status, cudaStream_t st);
// `count` cores core + i*core_stride (each r2 x s, ld) -> sigma + i*sigma_stride,
// status[i]; one CTA each (requires core_sigma_fits_cta).
bool core_sigma_fits_cta(int r2, int s);
cudaError_t launch_core_sigma_batched(const double* core, int r2, int s, int64_t ld,
                                      int64_t core_stride, int count, double* sigma,
                                      int64_t sigma_stride, int* status, cudaStream_t st,
                                      const int* active = nullptr, int cert_r1 = 0,
                                      float cert_ratio = 0.f);

// Device read-off (step 8).  Writes DevReadoff to `out`.
struct DevReadoff {
    int rank;        // -1 when not converged
    int gap_index;
    double gap_ratio;
    double tau;
    int status;
    int sweeps;      // Jacobi sweeps of the small-core step (status_in[2])
};
cudaError_t launch_readoff(const double* sigma, int r1, double scale, double eps, double norm_a,
                           const int* status_in, DevReadoff* out, double* sigma_scaled,
                           cudaStream_t st);

// ---- sketch-size proposal network (mlp.cu) -----------------------------------
constexpr int kMlpIn = 18, kMlpHidden = 128, kMlpOut = 12;
constexpr int kMlpParams = kMlpHidden * kMlpIn + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpOut * kMlpHidden + kMlpOut;
// logits (count x 12); keep (count x 256 activations) may be NULL for inference
cudaError_t mlp_forward(const float* P, const float* X, int count, float* logits, float* keep, cudaStream_t st);
// G += d(mean cross-entropy)/dP; *loss += mean loss
cudaError_t mlp_backward(const float* P, const float* X, const int* y, int count, const float* logits,
                         const float* keep, float* G, float* loss, cudaStream_t st);
cudaError_t mlp_adam(float* P, const float* G, float* M, float* V, float lr, int step, float wd, cudaStream_t st);
cudaError_t mlp_argmax(const float* logits, int count, int* cls, cudaStream_t st);
cudaError_t mlp_features(const double* sigma16, double eps, int64_t rows, int64_t cols, float* f, cudaStream_t st);
void mlp_init_host(float* P, uint64_t seed);

// ---- Algorithm 3 after the sketch (rangefinder.cu) ----------------------------
struct QbSelect {
    int r;           // selected target rank, -1 when no r in [0, r1] meets the criterion
    int met;         // r >= 0 and r + p <= s
    double bound;    // (1 + r/(p-1))^{1/2} (sum_{j>r} sigma^_j^2)^{1/2} at r
    double norm_a;   // ||A|| used (sigma^_1 unless given)
};
// Step 5 on the r1 trusted scaled sigma (device) of the width-s sketch; n = the
// smaller dimension (the conservative tail runs to it).
cudaError_t launch_select_rank(const double* sigma_scaled, int r1, int64_t n, double eps, double norm_a, int p,
                               int s, QbSelect* out, cudaStream_t st);
size_t qb_workspace_bytes(int64_t rows, int64_t cols, int k, bool tensor);
// Steps 7-8 for the first k columns of AX (rows x ldax FP32) with the FP64 core
// (r2 rows, ld_core) as the preconditioning sketch, in three stream-ordered
// stages on the workspace ws (qb_workspace_bytes(rows, cols, k)):
//   precondition:   W = A X_k R_s^{-1}, R_s from the core's Gram (FP64);
//   orthonormalise: two Cholesky-QR passes on W, Q (rows x k, ldq) with
//                   orthonormal columns;
//   product:        B = Q^T A_oriented (k x cols, ldb).
// *floored (device) is set when a Cholesky pivot had to be raised (an exactly
// singular Gram matrix).  launches (may be null) counts the kernels launched.
// AX(r, l) at AX[r sar + l sak] (sak == 1: row-major; sar == 1: transposed planes)
// tensor (with a non-null err_flag for the bounded waits): the Gram matrices V^T V
// and the products by (L^-1)^T on the tensor cores (both factors in three BF16
// terms, six products), where the operands suit those kernels; else CUDA cores.
cudaError_t launch_qb_precondition(const float* AX, int64_t sar, int64_t sak, int64_t rows, int64_t cols,
                                   const double* core, int64_t ld_core, int r2, int k, void* ws, int* floored,
                                   cudaStream_t st, int* launches, bool tensor = false, int* err_flag = nullptr);
cudaError_t launch_qb_orthonormalise(int64_t rows, int64_t cols, int k, float* Q, int64_t ldq, void* ws,
                                     int* floored, cudaStream_t st, int* launches, bool tensor = false,
                                     int* err_flag = nullptr);
// tensor: B = Q^T A on the tensor cores (qb_tc.cu) when the view allows it (else
// CUDA cores); err_flag receives a bounded wait's expiry.
cudaError_t launch_qb_product(const MatView& A, const float* Q, int64_t ldq, int k, float* B, int64_t ldb, void* ws,
                              bool tensor, int* err_flag, cudaStream_t st, int* launches);
// out (M x N, pitch ldo) = the sum over `splits` FP32 partials (pitch N, M N apart),
// added in FP64 in split order.
cudaError_t reduce_parts_f32(const float* part, int splits, int64_t M, int64_t N, float* out, int64_t ldo,
                             cudaStream_t st);
cudaError_t reduce_parts_f64(const float* part, int splits, int64_t M, int64_t N, double* out, int64_t ldo,
                             cudaStream_t st);

// ---- B = Q^T A on tcgen05 (qb_tc.cu) -------------------------------------------
bool qb_tc_supported(const MatView& A);
int64_t qb_tc_qt_ld(int64_t M);          // row pitch of the Q^T terms
int qb_tc_qt_rows(int k);                // rows per term (k rounded up to 128)
int qb_tc_splits(int64_t tiles, int64_t kchunks, int cap);
// Qt (3 x qb_tc_qt_rows(k) rows of pitch qb_tc_qt_ld(M), BF16 bits) = the three
// BF16 terms of Q^T (Q: M x k FP32, pitch ldq)
cudaError_t launch_qt_split(const float* Q, int64_t ldq, int64_t M, int k, uint16_t* Qt, cudaStream_t st);
// rows [c0, c0 + kq) of Q^T A (kq <= 128) into out (pitch ldo); split partials in
// part.  With out64, the partials are summed into out64 (FP64, pitch ldo64) instead.
cudaError_t launch_qb_product_tc(const MatView& A, const uint16_t* Qt, int k, int c0, int kq, float* out,
                                 int64_t ldo, float* part, int splits, int* err_flag, cudaStream_t st,
                                 double* out64 = nullptr, int64_t ldo64 = 0);
// Xt (3 planes of nrows rows, pitch ldt, BF16 bits) = the three BF16 terms of rows
// c0 .. c0+w-1 of S (FP32, pitch lds, cols columns), zero elsewhere: the X^T
// operand of launch_right_tc (xterms = 3) for X = S^T restricted to those columns.
cudaError_t launch_rows_split3(const float* S, int64_t lds, int c0, int w, int cols, int nrows, int64_t ldt,
                               uint16_t* Xt, cudaStream_t st);

// ---- batched estimate (batched.cu) --------------------------------------------
struct BatchedState;
// Level-synchronous batched Algorithm 1 (FP32 input, Gaussian X and Y); state is
// created on first use and owned by the handle.  launches is incremented by the
// number of kernels in one replay of the captured graph.  Exactly one of blocks
// (stored matrices) and kblocks (matrix-free kernel blocks, tensor-core
// precision only) is non-null.
int batched_estimate(BatchedState** st, const re_opts& o, const re_block* blocks, const re_kblock* kblocks,
                     int count, double eps, uint64_t seed, double* sigma_out, int sigma_cap, re_result* out,
                     cudaStream_t stream, int64_t* launches);
void batched_destroy(BatchedState* st);

}  // namespace re
