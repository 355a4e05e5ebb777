"""Checks of a rank estimate against the FP64 oracle where the spectrum has no
clear gap (test infrastructure, imported by the test files).

On a clear gap the GPU's rank must equal the oracle's.  Without one, a sketched
singular value can sit so close to the threshold tau = eps * sigma^_1 that the
GPU's rounding legitimately decides the other way.  `decision_consistent`
accepts a different answer only where the oracle's own sketched values put a
decision within the error the same test measured: band = 4 x the largest
|sigma^_gpu - sigma^_oracle| over the trusted values at the GPU's final width,
never wider than tau / 2.  Every ladder width up to the later of the two final
widths is checked the same way (Algorithm 1 step 8 at each width).

`desiderata_hold` is the Sec. 1.1 statement of what an eps-rank estimate should
satisfy, checked against the exact singular values of A:
sigma_{r+1}(A) < 10 eps ||A|| and, for r > 0, sigma_r(A) > 0.1 eps ||A||.
"""
from __future__ import annotations

import numpy as np

from oracle import algorithm1 as alg


def oracle_ladder(A, eps, kind, seed, s0=8, s_max=512, upto=None):
    """Oracle sketched values (trusted prefix) and read-off at every ladder width
    s0, 2 s0, ... up to `upto` (or the oracle's own final width)."""
    Ao, _ = alg.orient(np.asarray(A, dtype=np.float64))
    m, n = Ao.shape
    cap = alg.ladder_limits(m, n, kind, s_max)
    out = []
    s = s0
    while True:
        r1 = alg.r1_of_s(s)
        sig = alg.sketched_sigma(Ao, s, kind, seed)[:r1]
        ro = alg.readoff(sig, eps)
        out.append((s, sig, ro))
        last = (upto is None and ro.rank is not None) or 2 * s > cap or r1 >= n
        if (upto is not None and s >= upto) or (upto is None and last):
            break
        if 2 * s > cap:
            break
        s *= 2
    return out


def decision_consistent(rank, final_s, sig_gpu, A, eps, kind, seed, s0=8, s_max=512,
                        converged=True, err_floor=0.0):
    """True when the GPU's (rank, final width) follows from the oracle's sketched
    values up to decisions within the measured error band (see module doc)."""
    orc = alg.rank_estimate(np.asarray(A, dtype=np.float64), eps, kind=kind, seed=seed, s0=s0, s_max=s_max)
    lad = oracle_ladder(A, eps, kind, seed, s0, s_max, upto=max(final_s, orc.final_s))
    by_s = {s: (sig, ro) for s, sig, ro in lad}
    if final_s not in by_s:
        return False
    sig_o, ro_f = by_s[final_s]
    k = min(len(sig_o), len(sig_gpu))
    err = float(np.max(np.abs(np.asarray(sig_gpu[:k]) - sig_o[:k]))) if k else 0.0
    err = max(err, err_floor)

    def near(sig, ro):
        band = min(4.0 * err, 0.5 * ro.tau)
        return bool(np.any(np.abs(sig - ro.tau) <= band))

    # widths before the GPU's last: the GPU did not converge there
    for s, sig, ro in lad:
        if s >= final_s:
            break
        if ro.rank is not None and not near(sig, ro):
            return False
    if not converged:
        return ro_f.rank is None or near(sig_o, ro_f)
    if ro_f.rank is None:
        return near(sig_o, ro_f)
    if rank == ro_f.rank:
        return True
    band = min(4.0 * err, 0.5 * ro_f.tau)
    lo, hi = min(rank, ro_f.rank), max(rank, ro_f.rank)
    # every value between the two decisions must be within the band of tau
    return bool(np.all(np.abs(sig_o[lo:hi + 1][:max(hi - lo, 1)] - ro_f.tau) <= band))


def desiderata_hold(rank, A, eps, sigma_exact=None):
    """Sec. 1.1: sigma_{r+1} < 10 eps ||A|| and (r > 0) sigma_r > 0.1 eps ||A||."""
    s = np.linalg.svd(np.asarray(A, dtype=np.float64), compute_uv=False) if sigma_exact is None \
        else np.asarray(sigma_exact, dtype=np.float64)
    if s[0] == 0.0:
        return rank == 0
    thr = eps * s[0]
    ok_hi = rank >= len(s) or s[rank] < 10.0 * thr
    ok_lo = rank == 0 or s[rank - 1] > 0.1 * thr
    return bool(ok_hi and ok_lo)
