"""Pins for the oracle's generator (CPU only): published known answers,
library routines and distributional facts the paper relies on."""
import numpy as np
import pytest
import scipy.linalg
import scipy.stats

from oracle import rng


def test_philox_known_answers(golden):
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        c = [int(x, 16) for x in r[:4]]
        k = [int(x, 16) for x in r[4:6]]
        want = [int(x, 16) for x in r[6:10]]
        got = [int(v[()]) for v in rng.philox4x32_10(*c, *k)]
        assert got == want


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(50)
    out = rng.philox4x32_10(c0, 7, 3, 0, 11, 13)
    for i in (0, 17, 49):
        one = rng.philox4x32_10(i, 7, 3, 0, 11, 13)
        assert [int(o[i]) for o in out] == [int(v[()]) for v in one]


def test_ln_against_library():
    u = np.concatenate([np.float32(2.0 ** -24) * np.arange(1, 2000, dtype=np.float32),
                        np.linspace(1e-6, 1.0, 200001, dtype=np.float32)])
    got = rng.ln_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) < 2e-7
    assert rng.ln_f32(np.float32([1.0]))[0] == 0.0


def test_sincos_against_library():
    th = np.linspace(0, np.pi / 2, 200001, endpoint=False).astype(np.float32)
    s, c = rng.sincos_quarter_f32(th)
    assert np.max(np.abs(s - np.sin(th.astype(np.float64)))) < 3e-7
    assert np.max(np.abs(c - np.cos(th.astype(np.float64)))) < 3e-7


def test_normals_are_exact_bf16_and_fp16():
    z = rng.gaussian_x(512, 64, seed=5).ravel().astype(np.float32)
    assert np.array_equal(rng.round_normal(z), z)
    assert np.array_equal(z.astype(np.float16).astype(np.float32), z)
    # 16-bit fixed point: integer multiples of 2^-13 below 6 in magnitude
    k = z.astype(np.float64) * 8192.0
    assert np.array_equal(k, np.round(k)) and np.max(np.abs(z)) < 6.0
    nz = z[z != 0]
    assert np.min(np.abs(nz)) >= 2.0 ** -13


def _bits(x):
    return np.asarray(x, dtype=np.float32).view(np.uint32)


def test_bf16_rounding_ties_to_even():
    """Hand-chosen ties and near-ties: truncation, round-half-up or
    round-half-away would each get one of these wrong."""
    cases = [(0x3F808000, 0x3F800000),    # 1 + 2^-8: tie, even neighbour 1.0 below
             (0x3F818000, 0x3F820000),    # 1 + 3 2^-8: tie, even neighbour above
             (0x3F807FFF, 0x3F800000),    # just below the tie
             (0x3F808001, 0x3F810000),    # just above the tie
             (0xBF808000, 0xBF800000),    # -(1 + 2^-8): tie, magnitude down
             (0xBF818000, 0xBF820000),    # -(1 + 3 2^-8): tie, magnitude up
             (0x477F8000, 0x47800000)]    # 65280 + 128: tie, carries into the exponent
    src = np.array([c[0] for c in cases], dtype=np.uint32).view(np.float32)
    want = np.array([c[1] for c in cases], dtype=np.uint32)
    assert np.array_equal(_bits(rng.round_bf16(src)), want)


def test_grid_rounding_ties_to_even():
    """Below 2^-6 the normal goes to the 2^-13 grid, ties to the even multiple;
    zero comes out as +0; from 2^-6 on nothing moves."""
    u = 2.0 ** -13
    src = np.array([0.5 * u, 1.5 * u, 2.5 * u, 0.75 * u, -0.5 * u, -1.5 * u, -0.25 * u,
                    2.0 ** -6, -(2.0 ** -6) * 1.5, 3.0], dtype=np.float32)
    want = np.array([0.0, 2 * u, 2 * u, u, 0.0, -2 * u, 0.0, 2.0 ** -6, -(2.0 ** -6) * 1.5, 3.0],
                    dtype=np.float32)
    got = rng.round_normal(src)
    assert np.array_equal(_bits(got), _bits(want))      # bitwise: the zeros are +0


def test_normal_distribution():
    # 2^20 draws: moments and a Kolmogorov-Smirnov distance against N(0,1);
    # BF16 rounding moves a value by <= 2^-9 relative, which shifts the CDF by
    # < 2e-3, far below the KS threshold used.
    z = rng.gaussian_x(4096, 256, seed=1234).ravel()
    n = z.size
    assert abs(z.mean()) < 5.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 6.0 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 0.05
    ks = scipy.stats.kstest(z, "norm").statistic
    assert ks < 3e-3
    zy = rng.gaussian_y(64, 4096, seed=99).ravel()
    assert abs(zy.mean()) < 5.0 / np.sqrt(zy.size) and abs(zy.var() - 1) < 0.02


def test_gaussian_columns_are_prefix_consistent():
    a = rng.gaussian_x(100, 32, seed=3)
    b = rng.gaussian_x(100, 8, seed=3, col0=12)
    assert np.array_equal(a[:, 12:20], b)
    y = rng.gaussian_y(40, 77, seed=3)
    y2 = rng.gaussian_y(10, 77, seed=3, row0=21)
    assert np.array_equal(y[21:31], y2)
    assert not np.array_equal(rng.gaussian_x(10, 8, seed=4), rng.gaussian_x(10, 8, seed=3))


def test_marchenko_pastur_bounds_on_generated_matrix():
    # Theorem 3 (Eq. MP and DS): singular values of a 2000 x 500 standard Gaussian
    # lie in [sqrt(m)-sqrt(n)-t, sqrt(m)+sqrt(n)+t] except with prob 2 e^{-t^2/2}.
    m, n = 2000, 500
    G = rng.gaussian_x(m, n, seed=2024)
    sv = np.linalg.svd(G, compute_uv=False)
    t = 3.0
    assert sv[-1] >= np.sqrt(m) - np.sqrt(n) - t
    assert sv[0] <= np.sqrt(m) + np.sqrt(n) + t
    # and the bulk edges are approached (not a degenerate generator)
    assert sv[0] > np.sqrt(m) + np.sqrt(n) - 2 and sv[-1] < np.sqrt(m) - np.sqrt(n) + 2


@pytest.mark.parametrize("bits", list(range(0, 17)))
def test_feistel_is_a_bijection(bits):
    x = np.arange(1 << bits)
    p = rng.feistel_perm(x, bits, rng.STREAM_PX, seed=77)
    assert np.array_equal(np.sort(p), x)


def test_feistel_is_random_looking():
    p = rng.feistel_perm(np.arange(1 << 12), 12, rng.STREAM_PX, seed=1)
    assert np.sum(p == np.arange(1 << 12)) < 10
    q = rng.feistel_perm(np.arange(1 << 12), 12, rng.STREAM_PY, seed=1)
    assert not np.array_equal(p, q)


def test_signs_balanced():
    d = rng.signs(1 << 16, rng.STREAM_DX, seed=8)
    assert set(np.unique(d)) == {-1.0, 1.0}
    assert abs(d.mean()) < 5.0 / np.sqrt(d.size)


@pytest.mark.parametrize("n", [1, 2, 8, 64, 1024])
def test_hadamard_entries_match_sylvester(n):
    H = scipy.linalg.hadamard(n)
    got = rng.hadamard_entries(np.arange(n), np.arange(n))
    assert np.array_equal(got, H)


def test_srtt_full_sampling_is_orthogonal():
    # With every Hadamard column sampled, X = D H P (P a permutation), so
    # X^T X = n I and sigma(A X)/sqrt(n) = sigma(A) (Eq. Theta with r = n).
    n = 256
    X = rng.srtt_x(n, n, seed=11)
    assert np.array_equal(X.T @ X, n * np.eye(n))
    A = np.random.default_rng(0).standard_normal((300, n))
    sa = np.linalg.svd(A, compute_uv=False)
    sx = np.linalg.svd(A @ X, compute_uv=False) / np.sqrt(n)
    assert np.allclose(sa, sx, rtol=1e-12)
    Y = rng.srtt_y(128, 128, seed=11)
    assert np.array_equal(Y @ Y.T, 128 * np.eye(128))


def test_srtt_padding_drops_rows():
    # n not a power of two: X is the first n rows of the padded embedding.
    Xp = rng.srtt_x(64, 16, seed=2)
    # the same column indices, same signs for the first 40 rows
    X = rng.srtt_x(40, 16, seed=2)
    b40, b64 = rng.next_pow2_bits(40), rng.next_pow2_bits(64)
    assert b40 == b64 == 6
    assert np.array_equal(Xp[:40], X)


# ---------------------------------------------------------------------------
# HRTT (Sec. 3.4): X = D H C^T with a CountSketch C
def _countsketch(n_pad, s, seed):
    """C (s x n_pad) built directly: hash h(c) = pi^{-1}(c) mod s from an
    explicitly inverted permutation table, signs sigma_c of stream SX."""
    b = rng.next_pow2_bits(n_pad)
    perm = rng.feistel_perm(np.arange(n_pad), b, rng.STREAM_PX, seed)
    inv = np.argsort(perm)                       # inv[c] = q with pi(q) = c
    sigma = rng.signs(n_pad, rng.STREAM_SX, seed)
    C = np.zeros((s, n_pad))
    for c in range(n_pad):
        C[inv[c] % s, c] = sigma[c]
    return C


@pytest.mark.parametrize("n,s", [(256, 16), (100, 24), (300, 512), (64, 64), (1, 1)])
def test_hrtt_matches_explicit_countsketch(n, s):
    n_pad = 1 << rng.next_pow2_bits(n)
    C = _countsketch(n_pad, s, seed=21)
    assert np.array_equal(np.abs(C).sum(axis=0), np.ones(n_pad))   # one nonzero per column
    d = rng.signs(n, rng.STREAM_DX, seed=21)
    want = d[:, None] * (scipy.linalg.hadamard(n_pad)[:n].astype(np.float64) @ C.T)
    assert np.array_equal(rng.hrtt_x(n, s, seed=21), want)


def test_hrtt_full_width_is_signed_srtt():
    # s = n_pad: every bucket holds the single coordinate pi(k), so the HRTT is the
    # fully sampled SRTT with column k multiplied by sigma_{pi(k)}.
    n = 200
    n_pad = 256
    cols = rng.feistel_perm(np.arange(n_pad), 8, rng.STREAM_PX, seed=4)
    sigma = rng.signs(n_pad, rng.STREAM_SX, seed=4)
    assert np.array_equal(rng.hrtt_x(n, n_pad, seed=4), rng.srtt_x(n, n_pad, seed=4) * sigma[cols][None, :])


@pytest.mark.parametrize("s", [2, 16, 128])
def test_hrtt_buckets_fold(s):
    # h_{s/2}(c) = h_s(c) mod s/2: bucket k at width s/2 is buckets k and k + s/2 at s
    X = rng.hrtt_x(700, s, seed=9)
    Xh = rng.hrtt_x(700, s // 2, seed=9)
    assert np.array_equal(Xh, X[:, : s // 2] + X[:, s // 2:])


@pytest.mark.parametrize("s", [24, 64])
def test_hrtt_gram_closed_form(s):
    # n = n_pad: X^T X = C H D D H C^T = n_pad C C^T = n_pad diag(|bucket k|),
    # |bucket k| = number of q < n_pad with q = k mod s.
    n = 256
    X = rng.hrtt_x(n, s, seed=12)
    sizes = np.array([len(range(k, n, s)) for k in range(s)], dtype=np.float64)
    assert np.array_equal(X.T @ X, n * np.diag(sizes))


def test_hrtt_is_unbiased():
    # E[X X^T] = D H E[C^T C] H D = n_pad I (the signs sigma make E[C^T C] = I).
    # Averaged over 400 seeds each entry of X X^T / n_pad has standard deviation
    # about sqrt(2 / (s 400)) = 0.018 (s = 16): 0.1 is > 5 sigma.
    n, s = 32, 16
    acc = np.zeros((n, n))
    for seed in range(400):
        X = rng.hrtt_x(n, s, seed=seed)
        acc += X @ X.T / n
    acc /= 400
    assert np.max(np.abs(acc - np.eye(n))) < 0.1
    # without the signs sigma the diagonal of row 0 would be n_pad / s = 2
    assert abs(acc[0, 0] - 1.0) < 0.1


def test_hrtt_selected_rows():
    idx = np.array([0, 5, 99, 37])
    assert np.array_equal(rng.hrtt_x(100, 24, seed=3, rows=idx), rng.hrtt_x(100, 24, seed=3)[idx])


def test_hrtt_argument_errors():
    with pytest.raises(ValueError):
        rng.hrtt_x(100, 256, seed=0)                # s > n_pad = 128: empty buckets
    with pytest.raises(ValueError):
        rng.hrtt_x(100, 0, seed=0)


def test_hadamard_entries_wide_indices():
    # indices above 16 bits use both halves of the parity table: compare with the
    # Sylvester recursion H_{2N} = [[H, H], [H, -H]] at index 2^20 + i
    i = np.arange(0, 1 << 21, 4099)
    c = np.array([1 << 20, (1 << 20) | 5, 65537, 3])
    got = rng.hadamard_entries(i, c)
    want = np.array([[(-1.0) ** bin(int(a) & int(b)).count("1") for b in c] for a in i])
    assert np.array_equal(got, want)
