"""The rank checker of the GPU tests (tests/rankcheck.py) on the CPU: it must
accept the oracle's own answer and reject an answer one off, on the ungapped
kernel-block workload where the GPU tests use it (Sec. 1 structured blocks,
eps = 1e-6), and the Sec. 1.1 desiderata must hold for the oracle's rank."""
import numpy as np
import pytest

from oracle import algorithm1 as alg
from paper_2105_07388_gb300 import workloads as wl

from rankcheck import decision_consistent, desiderata_hold


@pytest.mark.parametrize("m,n,seed", [(300, 256, 100), (257, 400, 101), (512, 300, 302)])
def test_checker_rejects_off_by_one(m, n, seed):
    A = wl.kernel_block(m, n, seed=seed).double().numpy()
    orc = alg.rank_estimate(A, 1e-6, kind=alg.GAUSSIAN, seed=7, s_max=128)
    assert orc.converged
    # a GPU-like answer: the oracle's values with a relative error of 1e-9 sigma_1
    noise = 1e-9 * orc.sigma[0] * np.random.default_rng(seed).standard_normal(len(orc.sigma))
    sig = orc.sigma + noise
    assert decision_consistent(orc.rank, orc.final_s, sig, A, 1e-6, alg.GAUSSIAN, 7, s_max=128)
    for bad in (orc.rank - 1, orc.rank + 1):
        assert not decision_consistent(bad, orc.final_s, sig, A, 1e-6, alg.GAUSSIAN, 7, s_max=128)
    # stopping one width late is rejected too (values of that width, same error)
    s2 = 2 * orc.final_s
    sig2 = alg.sketched_sigma(A if A.shape[0] >= A.shape[1] else A.T, s2, alg.GAUSSIAN, 7)[:alg.r1_of_s(s2)]
    sig2 = sig2 + 1e-9 * orc.sigma[0]
    assert not decision_consistent(orc.rank, s2, sig2, A, 1e-6, alg.GAUSSIAN, 7, s_max=128)
    assert desiderata_hold(orc.rank, A, 1e-6)


def test_checker_band_follows_measured_error():
    """With an error as large as the distance of the nearest value to tau the
    other decision becomes acceptable; the band never exceeds tau / 2."""
    A = wl.kernel_block(300, 256, seed=100).double().numpy()
    orc = alg.rank_estimate(A, 1e-6, kind=alg.GAUSSIAN, seed=7, s_max=128)
    tau = 1e-6 * orc.sigma[0]
    d = abs(orc.sigma[orc.rank] - tau)           # first trusted value at or below tau
    if d >= 0.5 * tau:
        pytest.skip("no value near tau for this draw")
    sig = orc.sigma.copy()
    sig[0] += d / 3.0                           # measured error d/3: band 4d/3 covers it
    assert decision_consistent(orc.rank + 1, orc.final_s, sig, A, 1e-6, alg.GAUSSIAN, 7, s_max=128)


def test_desiderata_closed_form():
    A = np.diag([1.0, 1e-2, 1e-5, 1e-7, 1e-9])   # eps = 1e-6: 10 eps = 1e-5, 0.1 eps = 1e-7
    assert desiderata_hold(3, A, 1e-6)           # sigma_4 = 1e-7 < 1e-5 and sigma_3 = 1e-5 > 1e-7
    assert not desiderata_hold(2, A, 1e-6)       # sigma_3 = 1e-5 is not below 1e-5
    assert not desiderata_hold(4, A, 1e-6)       # sigma_4 = 1e-7 is not above 1e-7
    assert not desiderata_hold(1, A, 1e-6)
    assert desiderata_hold(0, np.zeros((3, 3)), 1e-6)
