"""Pins of the Algorithm 3 oracle (rank estimation + randomized rangefinder,
Sec. 5.1) against closed forms and published bounds."""
import math

import numpy as np
import pytest

from oracle import algorithm1 as alg
from oracle import algorithm3 as a3
from paper_2105_07388_gb300 import workloads as wl


def test_selection_exact_low_rank():
    # sigma^ = (1 x 5, 0 x 9), nothing beyond: the tail after r = 5 is exactly 0,
    # the tail after r = 4 is at least 1 > eps, for any p
    sig = np.array([1.0] * 5 + [0.0] * 9)
    for p in (2, 5, 10):
        assert a3.select_rank(sig, 14, 1e-3, p) == 5
    assert a3.select_rank(np.zeros(7), 100, 1e-3, 5) == 0       # A = 0: nothing to capture


def test_selection_geometric_closed_form():
    # sigma^_j = q^(j-1), j = 1..r1 and the tail extended by (n - r1) copies of q^(r1-1):
    # sum_{j>r} = q^(2r) (1 - q^(2(r1-r))) / (1 - q^2) + (n - r1) q^(2(r1-1))
    q, r1, n, p, eps = 0.7, 29, 40, 5, 1e-3
    sig = q ** np.arange(r1)
    want = None
    for r in range(r1 + 1):
        tail = q ** (2 * r) * (1 - q ** (2 * (r1 - r))) / (1 - q * q) + (n - r1) * q ** (2 * (r1 - 1))
        if math.sqrt(1 + r / (p - 1)) * math.sqrt(tail) <= eps:
            want = r
            break
    assert want is not None
    assert a3.select_rank(sig, n, eps, p) == want
    # the criterion with norm_a given uses it instead of sigma^_1
    assert a3.select_rank(sig * 2, n, eps, p, norm_a=2.0) == want


def test_selection_none_when_tail_too_heavy():
    sig = np.ones(7)
    assert a3.select_rank(sig, 1000, 1e-2, 5) is None


@pytest.fixture(scope="module")
def decaying():
    sig = wl.spectrum("fe", 300)                     # exponential decay, no gap
    A = wl.haar_matrix(500, 300, sig, seed=3).numpy()
    return A, sig.numpy()


def test_qb_factorization_invariants(decaying):
    A, s = decaying
    res = a3.qb(A, 1e-4, p=10, seed=2)
    Q, B = res.Q, res.B
    assert res.met and res.k == res.r + 10 and Q.shape == (500, res.k) and B.shape == (res.k, 300)
    assert np.max(np.abs(Q.T @ Q - np.eye(res.k))) < 1e-12
    # B = Q^T A, so ||A - QB||_F^2 = ||A||_F^2 - ||B||_F^2 (Pythagoras)
    e2 = np.linalg.norm(A - Q @ B) ** 2
    assert abs(e2 - (np.linalg.norm(A) ** 2 - np.linalg.norm(B) ** 2)) <= 1e-10 * np.linalg.norm(A) ** 2
    # no rank-k factorization beats the truncated SVD (Eckart-Young)
    assert math.sqrt(e2) >= math.sqrt(np.sum(s[res.k:] ** 2)) * (1 - 1e-9)


def test_qb_exact_low_rank():
    sig = wl.spectrum("step", 200, rank=12, tail_scale=0.0)
    A = wl.haar_matrix(400, 200, sig, seed=5).numpy()
    res = a3.qb(A, 1e-6, p=5, seed=1)
    assert res.met and res.r == 12 and res.k == 17
    assert np.linalg.norm(A - res.Q @ res.B) <= 1e-12 * np.linalg.norm(A)


def test_qb_halko_bound(decaying):
    # HMT Thm 10.5 (the paper's Eq. errRFfro1): E ||A - QB||_F <= (1 + r/(p-1))^{1/2}
    # (sum_{j>r} sigma_j^2)^{1/2} for a Gaussian X of r + p columns; the mean over
    # seeds of the ratio to the bound (true sigma, the r each run selected) is below 1
    A, s = decaying
    ratios = []
    for seed in range(12):
        res = a3.qb(A, 1e-3, p=5, seed=seed)
        bound = math.sqrt(1 + res.r / 4.0) * math.sqrt(np.sum(s[res.r:] ** 2))
        ratios.append(np.linalg.norm(A - res.Q @ res.B) / bound)
    assert np.mean(ratios) < 1.0, ratios


@pytest.mark.parametrize("fam,eps", [("fp", 1e-2), ("fp", 1e-4), ("se", 1e-1), ("fe", 1e-3)])
def test_qb_fixed_precision_goal(fam, eps):
    # the purpose of Algorithm 3: ||A - QB||_F <~ eps ||A|| with a near-minimal rank
    # (the criterion bounds an expectation, so a factor 2 is allowed)
    sig = wl.spectrum(fam, 300)
    A = wl.haar_matrix(600, 300, sig, seed=7).numpy()
    s = sig.numpy()
    for seed in range(4):
        res = a3.qb(A, eps, p=10, seed=seed)
        assert res.met
        err = np.linalg.norm(A - res.Q @ res.B)
        assert err <= 2.0 * eps * s[0], (fam, seed, err / (eps * s[0]))
        # near-minimal: the optimal rank-r error alone is not far below eps ||A||
        opt = math.sqrt(np.sum(s[res.r:] ** 2))
        assert opt <= 2.0 * eps * s[0]


def test_qb_transposed_and_errors():
    sig = wl.spectrum("step", 80, rank=9, tail_scale=1e-9)
    A = wl.haar_matrix(80, 200, sig, seed=4).numpy()          # m < n
    res = a3.qb(A, 1e-5, p=5, seed=3)
    assert res.transposed and res.r == 9 and res.Q.shape == (200, 14) and res.B.shape == (14, 80)
    assert np.linalg.norm(A.T - res.Q @ res.B) <= 1e-7 * np.linalg.norm(A)
    with pytest.raises(ValueError):
        a3.qb(A, 1e-5, p=1)
    with pytest.raises(ValueError):
        a3.qb(A, 0.0)


def test_qb_ladder_end_and_norm_override():
    # a full-rank matrix with a flat spectrum cannot meet eps = 1e-6 within s <= 32:
    # the ladder ends, k = s = 32 columns are returned and the criterion is not met
    A = np.random.default_rng(2).standard_normal((300, 200))
    res = a3.qb(A, 1e-6, p=5, seed=1, s_max=32)
    assert not res.met and res.final_s == 32 and res.k == 32 and res.r == 27
    assert np.max(np.abs(res.Q.T @ res.Q - np.eye(32))) < 1e-12
    # a larger ||A|| given by the caller loosens the criterion: a smaller or equal r
    sig = wl.spectrum("fp", 300)
    B = wl.haar_matrix(500, 300, sig, seed=2).numpy()
    r_default = a3.qb(B, 1e-3, p=5, seed=4).r
    r_loose = a3.qb(B, 1e-3, p=5, seed=4, norm_a=10.0 * float(sig[0])).r
    assert r_loose < r_default


def test_qb_sketch_wider_than_the_matrix():
    # n = 20 columns, sketch widths up to 32: A has only 20 singular values, so the
    # values beyond the 20th count as zero and r never exceeds n; the exact rank 20
    # meets any tolerance and k = min(r + p, n) = 20
    A = np.random.default_rng(3).standard_normal((200, 20))
    for eps in (1e-9, 1e-15):
        res = a3.qb(A, eps, p=5, seed=2)
        assert res.met and res.r == 20 and res.k == 20 and res.final_s == 32
    assert a3.select_rank(np.array([1.0, 0.5, 1e-15, 1e-15]), 2, 1e-16, 5) == 2
    assert np.linalg.norm(A - res.Q @ res.B) <= 1e-12 * np.linalg.norm(A)


def test_qb_met_when_the_sketch_covers_every_singular_value():
    # n = 450 < r1(512) = 465: the sketch holds all 450 singular values, r = 450 meets
    # any tolerance, and k = min(r + p, n) = 450 columns (not r + p = 550) factor A
    # exactly, so the criterion counts as met at s = 512 although r + p > s
    A = np.random.default_rng(5).standard_normal((600, 450))
    res = a3.qb(A, 1e-12, p=100, seed=4, s_max=512)
    assert res.met and res.r == 450 and res.k == 450 and res.final_s == 512
    assert np.linalg.norm(A - res.Q @ res.B) <= 1e-12 * np.linalg.norm(A)
