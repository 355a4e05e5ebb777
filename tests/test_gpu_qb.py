"""Algorithm 3 (rank estimation combined with the randomized rangefinder,
Sec. 5.1) through the C ABI against the FP64 oracle.

The oracle's thin QR is Householder; the library's is sketch-preconditioned
Cholesky-QR, so Q is compared through what is unique: the selected r, k and
width, orthonormality, B = Q^T A within the FP32 product bound, the
approximation error against the oracle's, and the span of the leading r
columns (the nested spans of A X_k's columns, fixed by the shared X)."""
import math

import numpy as np
import pytest
import torch

from oracle import algorithm3 as a3
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hd = rk.re_create(0)
    yield hd
    rk.re_destroy(hd)


def _sin_angle(Q1, Q2):
    """Sine of the largest principal angle between span(Q1) and span(Q2)."""
    c = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    return math.sqrt(max(0.0, 1.0 - float(c.min()) ** 2))


CASES = [
    ("step", 1500, 600, dict(rank=37, tail_scale=1e-9), 1e-5, 10),   # a clear gap
    ("fp", 1200, 500, {}, 1e-3, 10),                                # algebraic decay, no gap
    ("fe", 700, 700, {}, 1e-4, 5),                                   # exponential decay
    ("step", 400, 1100, dict(rank=20, tail_scale=1e-9), 1e-5, 5),   # m < n: A^T is factored
]


@pytest.fixture(scope="module")
def h_tc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    hd = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    yield hd
    rk.re_destroy(hd)


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("fam,m,n,kw,eps,p", CASES)
def test_qb_parity(h, h_tc, tensor, fam, m, n, kw, eps, p):
    """FP32 handle: CUDA-core products; BF16x3 handle: B = Q^T A on the tensor
    cores (both factors split into three BF16 terms, six products)."""
    sig = wl.spectrum(fam, min(m, n), **kw)
    A = wl.haar_matrix(m, n, sig, seed=m + n).numpy().astype(np.float32)
    A64 = A.astype(np.float64)
    res, Q, B = rk.re_rank_estimate_qb(h_tc if tensor else h, torch.from_numpy(A).cuda(), eps, p=p, seed=21)
    orc = a3.qb(A64, eps, p=p, seed=21)
    assert res.status == 0
    assert bool(res.flags & rk.RE_TRANSPOSED) == (m < n) == orc.transposed
    assert bool(res.flags & rk.RE_CONVERGED) == orc.met
    assert res.final_s == orc.final_s
    if fam == "step":
        assert res.r == orc.r == kw["rank"]
    else:
        # sketched sigma agree to 1e-4 sigma_1: at the threshold the choice may move by one
        assert abs(res.r - orc.r) <= 1
    assert res.k == res.r + p
    Qg, Bg = Q.double().cpu().numpy(), B.double().cpu().numpy()
    k = res.k
    assert np.max(np.abs(Qg.T @ Qg - np.eye(k))) < 1e-5
    Ao = A64.T if m < n else A64
    bound = 2.0 * (Ao.shape[0] / 32 + 32) * U32 * (np.abs(Qg).T @ np.abs(Ao)) + 1e-30
    assert np.all(np.abs(Bg - Qg.T @ Ao) <= bound)
    nrm = np.linalg.norm(Ao)
    err_g = np.linalg.norm(Ao - Qg @ Bg)
    err_o = np.linalg.norm(Ao - orc.Q @ orc.B)
    assert err_g <= 1.5 * err_o + 1e-5 * nrm, (err_g / nrm, err_o / nrm)
    r = min(res.r, orc.r)
    if r > 0:
        assert _sin_angle(Qg[:, :r], orc.Q[:, :r]) < 1e-2
    assert res.bound > 0 and res.bound <= eps * res.norm_a * (1 + 1e-12)


def test_qb_caller_buffers_with_any_row_pitch(h_tc):
    """Q and B given by the caller with row pitches that are not multiples of 4
    floats: the tensor-core Cholesky-QR works on its own padded buffers and copies
    the k columns of Q out, so the results equal those with the library's buffers
    and nothing past column k of Q's rows is written."""
    sig = wl.spectrum("step", 500, rank=150, tail_scale=1e-9)
    A = wl.haar_matrix(1200, 500, sig, seed=1700).to(torch.float32).cuda()
    res0, Q0, B0 = rk.re_rank_estimate_qb(h_tc, A, 1e-5, p=13, seed=21)
    k_cap = 500
    Qbuf = torch.full((1200, k_cap + 3), 7.0, dtype=torch.float32, device="cuda")
    Bbuf = torch.full((k_cap, 500 + 1), 7.0, dtype=torch.float32, device="cuda")
    res, Q, B = rk.re_rank_estimate_qb(h_tc, A, 1e-5, p=13, seed=21, Q=Qbuf[:, :k_cap], B=Bbuf[:, :500],
                                       k_cap=k_cap)
    assert (res.r, res.k, res.final_s, res.flags) == (res0.r, res0.k, res0.final_s, res0.flags)
    # k = 163: the tensor-core products run (k >= 64) on rows padded to 168 columns
    assert res.r == 150 and res.k == 163
    assert torch.equal(Q, Q0) and torch.equal(B, B0)
    # the columns past k of every row of Q, and the pitch padding, keep their contents
    assert bool((Qbuf[:, res.k:] == 7.0).all()) and bool((Bbuf[:, 500:] == 7.0).all())


def test_qb_exact_low_rank_and_zero(h):
    sig = wl.spectrum("step", 300, rank=12, tail_scale=0.0)
    A = wl.haar_matrix(700, 300, sig, seed=9).to(torch.float32).cuda()
    res, Q, B = rk.re_rank_estimate_qb(h, A, 1e-5, p=5, seed=3)
    assert res.r == 12 and res.k == 17 and res.flags & rk.RE_CONVERGED
    err = torch.linalg.norm(A.double() - Q.double() @ B.double()) / torch.linalg.norm(A.double())
    assert float(err) < 1e-5
    Z = torch.zeros(500, 200, device="cuda")
    res, Q, B = rk.re_rank_estimate_qb(h, Z, 1e-3, p=4, seed=1)
    assert res.r == 0 and res.k == 4
    assert torch.all(torch.isfinite(Q)) and torch.all(B == 0)


def test_qb_errors(h):
    A = torch.randn(300, 200, device="cuda")
    Q = torch.empty(300, 4, device="cuda")
    B = torch.empty(4, 200, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate_qb(h, A, 1e-3, p=5, seed=1, Q=Q, B=B, k_cap=4)      # full rank: k > 4
    assert e.value.code == rk.RE_ERR_ARG
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate_qb(h, A, 1e-3, p=1)
    assert e.value.code == rk.RE_ERR_ARG


@pytest.mark.parametrize("m,n,p,eps,s_max,final_s", [
    (200, 20, 5, 1e-9, 512, 32),       # r1(32) = 29 > n: the values beyond the 20th count as zero
    (200, 20, 5, 1e-15, 512, 32),
    (600, 450, 100, 1e-12, 512, 512),  # r + p = 550 > s, but k = min(r + p, n) = 450 <= s
])
def test_qb_sketch_wider_than_the_matrix(h, m, n, p, eps, s_max, final_s):
    """The step-5 selection once the sketch trusts more values than A has (n <
    r1): r = n meets any tolerance, k = min(r + p, n), as in the oracle."""
    A = np.random.default_rng(m + n).standard_normal((m, n)).astype(np.float32)
    A64 = A.astype(np.float64)
    res, Q, B = rk.re_rank_estimate_qb(h, torch.from_numpy(A).cuda(), eps, p=p, seed=2)
    orc = a3.qb(A64, eps, p=p, seed=2, s_max=s_max)
    assert orc.met and orc.r == n and orc.k == n and orc.final_s == final_s
    assert res.status == 0 and res.flags & rk.RE_CONVERGED
    assert (res.r, res.k, res.final_s) == (orc.r, orc.k, orc.final_s)
    Qg, Bg = Q.double().cpu().numpy(), B.double().cpu().numpy()
    nrm = np.linalg.norm(A64)
    assert np.linalg.norm(A64 - Qg @ Bg) <= 1e-5 * nrm
    assert np.linalg.norm(A64 - orc.Q @ orc.B) <= 1e-12 * nrm


@pytest.mark.parametrize("precision", [0, 1])
def test_qb_noise_floor_columns(precision):
    """The ladder ends at s_max with hundreds of columns of A X at the FP32 noise
    floor (eps below what the FP32 sketch resolves, while the FP64 oracle meets
    the criterion at s = 256): every column of Q stays finite,
    the columns that are not deflated are orthonormal, deflated ones are zero
    and flagged, and Q B approximates A as well as the oracle's factorization."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m, n = 8192, 2048
    sig = wl.spectrum("step", n, rank=200, tail_scale=1e-6)
    A = wl.householder_matrix(m, n, sig, seed=4, device="cuda").to(torch.float32)
    hd = rk.re_create(0, rk.make_opts(precision=precision))
    try:
        res, Q, B = rk.re_rank_estimate_qb(hd, A, 1e-6, p=10, seed=5)
    finally:
        rk.re_destroy(hd)
    assert res.status == 0 and res.flags & rk.RE_LOWER_BOUND_ONLY
    assert res.final_s == 512 and res.k == 512 and res.r == 502
    assert torch.all(torch.isfinite(Q)) and torch.all(torch.isfinite(B))
    Qg = Q.double()
    norms = torch.linalg.norm(Qg, dim=0)
    live = norms > 0.5
    assert torch.all(live | (norms == 0))
    assert bool(res.flags & rk.RE_QB_DEFLATED) == bool((~live).any())
    Ql = Qg[:, live]
    assert float((Ql.T @ Ql - torch.eye(Ql.shape[1], device=Ql.device, dtype=Ql.dtype)).abs().max()) < 1e-5
    A64 = A.double()
    nrm = float(torch.linalg.norm(A64))
    err_g = float(torch.linalg.norm(A64 - Qg @ B.double()))
    # the FP64 oracle resolves the tail and meets the criterion earlier (k = 210 at
    # s = 256); the GPU's wider factorization must approximate A at least as well
    orc = a3.qb(A64.cpu().numpy(), 1e-6, p=10, seed=5)
    assert orc.met and orc.k <= res.k
    err_o = float(np.linalg.norm(A64.cpu().numpy() - orc.Q @ orc.B))
    assert err_g <= 1.5 * err_o + 1e-5 * nrm, (err_g / nrm, err_o / nrm)


def test_qb_exact_product_ladder_meets_the_criterion():
    """With the exact-product sketch (RE_PREC_EXACT) the tail values that step 5
    sums are resolved: on the matrix where the FP32 ladder runs to s_max, the
    criterion is met at the oracle's r, k and width, and Q B approximates A as
    well as the oracle's factorization."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    m, n = 8192, 2048
    sig = wl.spectrum("step", n, rank=200, tail_scale=1e-6)
    A = wl.householder_matrix(m, n, sig, seed=4, device="cuda").to(torch.float32)
    hd = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_EXACT))
    try:
        res, Q, B = rk.re_rank_estimate_qb(hd, A, 1e-6, p=10, seed=5)
    finally:
        rk.re_destroy(hd)
    A64 = A.double()
    orc = a3.qb(A64.cpu().numpy(), 1e-6, p=10, seed=5)
    assert orc.met and res.flags & rk.RE_CONVERGED
    assert (res.r, res.k, res.final_s) == (orc.r, orc.k, orc.final_s) == (200, 210, 256)
    # the p extra columns sit at the 5e-9 tail: below what the FP64 Gram matrix of
    # the core (squared: 2.5e-17 < 2^-53) and the FP32 A X resolve, so they may
    # deflate; the r leading columns never do
    Qg = Q.double()
    norms = torch.linalg.norm(Qg, dim=0)
    live = norms > 0.5
    assert torch.all(live | (norms == 0)) and bool(live[:200].all())
    assert bool(res.flags & rk.RE_QB_DEFLATED) == bool((~live).any())
    Ql = Qg[:, live]
    assert float((Ql.T @ Ql - torch.eye(Ql.shape[1], device=Ql.device, dtype=Ql.dtype)).abs().max()) < 1e-5
    nrm = float(torch.linalg.norm(A64))
    err_g = float(torch.linalg.norm(A64 - Qg @ B.double()))
    err_o = float(np.linalg.norm(A64.cpu().numpy() - orc.Q @ orc.B))
    assert err_g <= 1.5 * err_o + 1e-5 * nrm, (err_g / nrm, err_o / nrm)
    assert res.bound <= 1e-6 * res.norm_a * (1 + 1e-12)
