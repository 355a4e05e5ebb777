"""Pins of the oracle's subsampled randomized DCT left embedding (Eq. (Theta)
with F the orthonormal DCT-II, coherence eta = 2; Sec. 4, the transform the
paper's experiments use for Y) against what the mathematics fixes."""
import math

import numpy as np
import pytest

from oracle import algorithm1 as alg
from oracle import rng


@pytest.mark.parametrize("N", [1, 2, 8, 64, 1024])
def test_dct_matrix_is_the_library_dct(N):
    """sqrt(N)^-1 dct_entries is scipy's orthonormal DCT-II applied to the identity."""
    scipy_fft = pytest.importorskip("scipy.fft")
    C = rng.dct_entries(np.arange(N), np.arange(N), N) / math.sqrt(N)
    R = scipy_fft.dct(np.eye(N), type=2, norm="ortho", axis=0)
    assert np.max(np.abs(C - R)) < 1e-13


@pytest.mark.parametrize("N", [4, 32, 256])
def test_dct_matrix_orthogonal_and_closed_form(N):
    C = rng.dct_entries(np.arange(N), np.arange(N), N)
    assert np.max(np.abs(C @ C.T - N * np.eye(N))) < 1e-10 * N
    assert np.all(C[0] == 1.0)                                  # frequency 0: constant
    # k = 1, i = 0: sqrt(2) cos(pi / (2N)); k = N/2, i = 0: sqrt(2) cos(pi/4) = 1
    assert abs(C[1, 0] - math.sqrt(2.0) * math.cos(math.pi / (2 * N))) < 1e-15
    assert abs(C[N // 2, 0] - 1.0) < 1e-14
    # eta = N max |F_ij|^2 <= 2 for the DCT (Sec. 4), reached as N grows: the
    # largest entry is sqrt(2) cos(pi / (2N)) (k = 1, i = 0)
    eta = np.max((C / math.sqrt(N)) ** 2) * N
    assert 2.0 * math.cos(math.pi / (2 * N)) ** 2 - 1e-12 <= eta <= 2.0


def test_phase_reduction_is_exact():
    """Large frequency-index products reduced modulo 4N give the same cosine as
    the unreduced angle evaluated in exact arithmetic (mpmath-free check through
    the symmetry cos(pi (2i+1) k / 2N) = cos(pi (2i+1) (k + 4N) / 2N))."""
    N = 1 << 20
    k = np.array([3, N - 1, N // 3])
    i = np.array([0, 1, N - 1, 12345])
    a = rng.dct_entries(k, i, N)
    b = rng.dct_entries(k + 4 * N, i, N)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("m", [64, 100])
def test_full_sampling_is_an_isometry(m):
    """All m_pad rows of Y = sqrt(m_pad) S F D with m = m_pad (every frequency once,
    the Feistel map a bijection) give Y^T Y = m_pad I; with zero padding (m < m_pad)
    the first m columns keep Y^T Y = m_pad I."""
    mp = 1 << rng.next_pow2_bits(m)
    Y = rng.srct_y(mp, m, 9)
    assert np.max(np.abs(Y.T @ Y - mp * np.eye(m))) < 1e-10 * mp


def test_rows_are_prefix_consistent_and_signed():
    Y = rng.srct_y(24, 200, 5)
    Y2 = rng.srct_y(16, 200, 5, row0=8)
    assert np.array_equal(Y[8:], Y2)
    d = rng.signs(200, rng.STREAM_DY, 5)
    k = rng.feistel_perm(np.arange(24), rng.next_pow2_bits(200), rng.STREAM_PY, 5)
    # undoing the signs leaves the plain DCT rows of the sampled frequencies
    assert np.array_equal(Y * d[None, :], rng.dct_entries(k, np.arange(200), 256))


def test_srct_left_sketch_embeds():
    """Sec. 4 (Corollary on Theta A X): sigma_i(Theta B) / sigma_i(B) within
    1 +- 0.5 for an incoherent m x 40 B with r2 = 320 rows (eta = 2)."""
    g = np.random.default_rng(2)
    B = np.linalg.qr(g.standard_normal((4096, 40)))[0] @ np.diag(np.logspace(0, -6, 40))
    TB = alg.left_sketch(B, 320, alg.GAUSSIAN, 11, ykind=alg.SRCT) / math.sqrt(320)
    ratio = np.linalg.svd(TB, compute_uv=False) / np.linalg.svd(B, compute_uv=False)
    assert np.all(ratio > 0.5) and np.all(ratio < 1.5)


def test_rank_estimate_with_srct_left_embedding():
    """Gaussian X with the SRCT Y: exact rank on a clear gap (1e-9 tail)."""
    g = np.random.default_rng(3)
    m, n, r = 600, 300, 25
    U = np.linalg.qr(g.standard_normal((m, n)))[0]
    V = np.linalg.qr(g.standard_normal((n, n)))[0]
    sig = np.where(np.arange(n) < r, 1.0, 1e-9)
    A = (U * sig) @ V.T
    res = alg.rank_estimate(A, 1e-5, kind=alg.GAUSSIAN, seed=4, ykind=alg.SRCT)
    assert res.converged and res.rank == r and res.final_s == 32


# ---- the hashed randomized DCT right embedding (Sec. 3.4; the paper's X in Sec. 6)

@pytest.mark.parametrize("n,s", [(64, 8), (100, 16), (256, 32)])
def test_hrct_columns_are_the_library_inverse_dct(n, s):
    """Column k of X is d * sqrt(N) * (inverse orthonormal DCT-II of the bucket's
    signed indicator): scipy's idct (type 2, orthonormal) of that vector."""
    scipy_fft = pytest.importorskip("scipy.fft")
    b = rng.next_pow2_bits(n)
    N = 1 << b
    X = rng.hrct_x(n, s, 23)
    d = rng.signs(n, rng.STREAM_DX, 23)
    sig = rng.signs(N, rng.STREAM_SX, 23)
    for k in range(s):
        v = np.zeros(N)
        c = rng.feistel_perm(np.arange(k, N, s), b, rng.STREAM_PX, 23)
        v[c] = sig[c]
        ref = d * math.sqrt(N) * scipy_fft.idct(v, type=2, norm="ortho")[:n]
        assert np.max(np.abs(X[:, k] - ref)) < 1e-10 * math.sqrt(N)


def test_hrct_full_width_is_an_isometry_and_folds():
    """s = n_pad (one coordinate per bucket): X^T X = n_pad I for n = n_pad.  Halving
    the width merges bucket k with bucket k + s/2: X_{s/2}[:, k] = X_s[:, k] + X_s[:, k + s/2]."""
    n = 128
    X = rng.hrct_x(n, n, 4)
    assert np.max(np.abs(X.T @ X - n * np.eye(n))) < 1e-9 * n
    X16, X8 = rng.hrct_x(200, 16, 4), rng.hrct_x(200, 8, 4)
    assert np.max(np.abs(X8 - (X16[:, :8] + X16[:, 8:]))) < 1e-12 * 16


def test_hrct_rank_on_a_diagonal_matrix():
    """Sec. 3.4 / Sec. 6: hashed embeddings keep the embedding on a diagonal (most
    coherent) matrix: the exact rank of a gapped diagonal spectrum, with Gaussian
    and with SRCT left embeddings."""
    n, r = 1024, 60
    sig = np.where(np.arange(n) < r, np.logspace(0, -1, n), 1e-10)
    A = np.diag(sig)
    for yk in (alg.GAUSSIAN, alg.SRCT):
        res = alg.rank_estimate(A, 1e-6, kind=alg.HRCT, seed=3, ykind=yk)
        assert res.converged and res.rank == r
