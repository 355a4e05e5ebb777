"""Hashed randomized DCT right embedding (Sec. 3.4 with the DCT-II, the X of the
paper's experiments, Sec. 6) on the GPU against the FP64 oracle.

X is generated densely in FP32 (each entry a compensated sum of its bucket's
cosines from an FP32 table) and enters the right sketch either as three exact
BF16 terms on the tensor cores or through the FP32 CUDA-core sketch.
"""
import math

import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from oracle import rng
from paper_2105_07388_gb300 import rankest as rk

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _handle(precision, **kw):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    return rk.re_create(0, rk.make_opts(precision=precision, **kw))


@pytest.fixture(scope="module")
def h32():
    hd = _handle(rk.RE_PREC_FP32)
    yield hd
    rk.re_destroy(hd)


@pytest.fixture(scope="module")
def htc():
    hd = _handle(rk.RE_PREC_BF16X3)
    yield hd
    rk.re_destroy(hd)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def _x_bound(n, s, X):
    """Per-entry bound of the FP32 X: each of the L = ceil(n_pad / s) terms carries
    the table's rounding (u |cos|) and the product by sqrt(2) (u), the compensated
    sum adds 2u |x| + O(L u^2) sum |terms|; with sum |terms| <= sqrt(2) L,
    |err| <= 2u |x| + 4u sqrt(2) L."""
    N = 1 << rng.next_pow2_bits(n)
    L = -(-N // s)
    return 2.0 * U32 * np.abs(X) + 4.0 * U32 * math.sqrt(2.0) * L


@pytest.mark.parametrize("n,s", [(1000, 64), (37, 24), (4099, 40), (256, 256), (3000, 8)])
def test_hrct_x_matches_oracle(h32, n, s):
    out = torch.empty(n, s, dtype=torch.float32, device="cuda")
    rk.re_embedding_x(h32, rk.RE_HRCT, 77, n, 0, s, out)
    X = rng.hrct_x(n, s, 77)
    err = np.abs(out.double().cpu().numpy() - X)
    assert np.all(err <= _x_bound(n, s, X)), float(np.max(err / _x_bound(n, s, X)))
    # the bucket folding of the definition holds on the device's X as well
    if s % 2 == 0 and s >= 16:
        half = torch.empty(n, s // 2, dtype=torch.float32, device="cuda")
        rk.re_embedding_x(h32, rk.RE_HRCT, 77, n, 0, s // 2, half)
        fold = (out[:, : s // 2].double() + out[:, s // 2:].double()).cpu().numpy()
        Xh = rng.hrct_x(n, s // 2, 77)
        xb = _x_bound(n, s, X)
        bound = _x_bound(n, s // 2, Xh) + xb[:, : s // 2] + xb[:, s // 2:]
        assert np.all(np.abs(half.double().cpu().numpy() - fold) <= bound)


def test_hrct_x_large_order_rows(h32):
    """2^15-point order (n = 20000): sampled rows against the oracle's rows."""
    n, s = 20000, 16
    out = torch.empty(n, s, dtype=torch.float32, device="cuda")
    rk.re_embedding_x(h32, rk.RE_HRCT, 5, n, 0, s, out)
    rows = np.random.default_rng(1).choice(n, 64, replace=False)
    rows = np.sort(np.append(rows, [0, n - 1]))
    X = rng.hrct_x(n, s, 5, rows=rows)
    err = np.abs(out.double().cpu().numpy()[rows] - X)
    assert np.all(err <= _x_bound(n, s, X))


def _sketch_bound(Ao, X, n, s):
    """|AX - A X_oracle| <= |A| |X_err| (the FP32 X) + the FP32 accumulation of
    |A| |X| (split-K partial sums, as for the Gaussian sketch)."""
    rows, cols = Ao.shape
    absA = np.abs(Ao)
    return absA @ _x_bound(n, s, X) + 2.0 * (cols / 16 + 32) * U32 * (absA @ np.abs(X)) + 1e-30


@pytest.mark.parametrize("m,n,s", [
    (3000, 2500, 64),       # one launch of 64 columns (N = 4096: buckets of 64)
    (2000, 1000, 200),      # two launches (128 + 72 columns), ragged MMA width
    (5003, 777, 24),        # odd row count, N = 1024
    (1100, 2300, 40),       # m < n: A^T (the CUDA-core sketch under both precisions)
    (4000, 4097, 8),        # row pitch not a multiple of 4, N = 8192
])
@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_hrct_right_sketch_parity(h32, htc, m, n, s, prec):
    hd = h32 if prec == "fp32" else htc
    A = np.random.default_rng(m * 7 + n + s).standard_normal((m, n)).astype(np.float32)
    Ad = dev(A)
    Ao, _ = alg.orient(A.astype(np.float64))
    rows, cols = Ao.shape
    AX = torch.zeros(rows, s, dtype=torch.float32, device="cuda")
    rk.re_sketch_apply(hd, Ad, 0, s, rk.RE_HRCT, 61, AX)
    X = alg.embeddings(alg.HRCT, cols, rows, s, 61, r2=0)[0]
    ref = Ao @ X
    err = np.abs(AX.double().cpu().numpy() - ref)
    bound = _sketch_bound(Ao, X, cols, s)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_hrct_core_parity(htc):
    """The whole width-s sketch and its 2s x s core (Gaussian Y) in one call."""
    m, n, s = 2000, 700, 32
    A = np.random.default_rng(8).standard_normal((m, n)).astype(np.float32)
    AX = torch.zeros(m, s, dtype=torch.float32, device="cuda")
    core = torch.zeros(2 * s, s, dtype=torch.float64, device="cuda")
    rk.re_sketch_apply(htc, dev(A), 0, s, rk.RE_HRCT, 31, AX, core)
    A64 = A.astype(np.float64)
    ref = alg.core(A64, s, alg.HRCT, 31)
    X, Y = alg.embeddings(alg.HRCT, n, m, s, 31)
    ax_err = _sketch_bound(A64, X, n, s)
    ax_abs = np.abs(A64) @ np.abs(X) + ax_err
    bound = np.abs(Y) @ ax_err + 4.0 * (m / 32 + 64) * U32 * (np.abs(Y) @ ax_abs)
    assert np.all(np.abs(core.cpu().numpy() - ref) <= bound)


@pytest.mark.parametrize("prec", [rk.RE_PREC_FP32, rk.RE_PREC_BF16X3])
@pytest.mark.parametrize("ykind", [rk.RE_GAUSSIAN, rk.RE_SRCT])
def test_hrct_rank_on_a_diagonal_matrix(prec, ykind):
    """Sec. 3.4 / Sec. 6: on a diagonal (maximally coherent) matrix with a gap the
    hashed DCT keeps the exact rank; the oracle's width, rank and sketched values
    (within 1e-4 sigma^_1) with the Gaussian and with the SRCT left embedding."""
    n, r = 1024, 60
    sig = np.where(np.arange(n) < r, np.logspace(0, -1, n), 1e-10)
    A = np.diag(sig)
    hd = _handle(prec, y_kind=ykind)
    try:
        res, sg = rk.re_rank_estimate(hd, dev(A), 1e-4, rk.RE_HRCT, 3, sigma_cap=512)
    finally:
        rk.re_destroy(hd)
    orc = alg.rank_estimate(A, 1e-4, kind=alg.HRCT, seed=3, ykind=ykind)
    assert orc.converged and orc.rank == r
    assert (res.rank, res.final_s, res.passes) == (orc.rank, orc.final_s, orc.passes)
    assert np.max(np.abs(sg[:res.n_sigma] - orc.sigma[:res.n_sigma])) <= 1e-4 * orc.sigma[0]


def test_hrct_errors(h32):
    A = torch.randn(300, 100, device="cuda")
    AX = torch.zeros(300, 256, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply(h32, A, 8, 8, rk.RE_HRCT, 1, AX)          # not appendable
    assert e.value.code == rk.RE_ERR_ARG
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply(h32, A, 0, 256, rk.RE_HRCT, 1, AX)        # s > n_pad = 128
    assert e.value.code == rk.RE_ERR_ARG
    out = torch.empty(100, 16, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_embedding_x(h32, rk.RE_HRCT, 1, 100, 8, 8, out)
    assert e.value.code == rk.RE_ERR_ARG
    with pytest.raises(rk.RankEstError) as e:
        rk.re_create(0, rk.make_opts(y_kind=rk.RE_HRCT))             # right embedding only
    assert e.value.code == rk.RE_ERR_ARG
    # full column rank 100: the read-off at s = 128 finds sigma_101 at the rounding level
    res, _ = rk.re_rank_estimate(h32, A, 1e-3, rk.RE_HRCT, 1)
    assert res.rank == 100 and res.flags & rk.RE_CONVERGED and res.final_s == 128
