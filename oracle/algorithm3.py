"""Algorithm 3 (Sec. 5.1, "Rank Estimation combined with Randomized Rangefinder")
in FP64 on the CPU.  TEST INFRASTRUCTURE ONLY (see the package docstring).

The steps in the algorithm box's order:

  1-3  Algorithm 1's sketches at width s (Gaussian X and Y, the reading of
       ``algorithm1``) and the first r1 sketched singular values   -> ``algorithm1.sketched_sigma``
  4    sigma^_i = sigma^_{r1} for r1 < i <= n (the conservative tail)  -> ``tail_sums``
  5    r = the smallest r with
           (1 + r/(p-1))^{1/2} (sum_{j>r} sigma^_j^2)^{1/2} <= eps ||A||
       (Halko, Martinsson & Tropp's Frobenius bound, Eq. errRFfro1, with the
       estimates in place of the singular values); if none exists, or r + p
       exceeds the columns sketched, grow the sketch by doubling  -> ``select_rank`` / ``qb``
  6    AX <- AX[:, :r+p]
  7    Q = thin QR of AX (Householder, LAPACK), columns signed so that R has a
       positive diagonal (then Q is unique)
  8    B = Q^T A

Readings taken here (the CUDA path takes the same ones):

* ||A|| is sigma^_1 unless the caller gives it (the algorithm's fallback).
* r ranges over 0 .. min(r1, n) (r = 0 when even the whole estimated tail is
  below eps ||A||); the tail beyond r1 counts n - r1 copies of sigma^_{r1}, n
  the smaller dimension, and sketched values beyond the n-th count as zero.
  k = min(r + p, n) must not exceed the width s; otherwise s doubles (when r + p
  exceeds n, the n columns of a sketch at least n wide already factor A).
* When the ladder cannot grow, the largest factorization it has (k = s, at
  most n) is returned with ``met = False`` and r = k - p.
* m < n: the factorization is of A^T (Q spans the column space of A^T).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import algorithm1 as alg
from . import rng


def tail_sums(sig_trusted: np.ndarray, n: int) -> np.ndarray:
    """Step 4: T[r] = sum_{j>r} sigma^_j^2 for r = 0 .. min(r1, n), with sigma^_j =
    sigma^_{r1} for r1 < j <= n; values beyond the n-th are zero (A has only n
    singular values), so a sketch wider than n trusts at most n of them."""
    sig = np.asarray(sig_trusted, dtype=np.float64)[:max(n, 0)]
    r1 = sig.size
    rest = max(n - r1, 0) * (sig[-1] ** 2 if r1 else 0.0)
    T = np.empty(r1 + 1)
    acc = rest
    T[r1] = acc
    for r in range(r1 - 1, -1, -1):
        acc += sig[r] ** 2
        T[r] = acc
    return T


def select_rank(sig_trusted: np.ndarray, n: int, eps: float, p: int,
                norm_a: float | None = None) -> int | None:
    """Step 5: the smallest r in [0, r1] meeting the Frobenius criterion, or None."""
    sig = np.asarray(sig_trusted, dtype=np.float64)
    ref = norm_a if (norm_a is not None and norm_a > 0) else (sig[0] if sig.size else 0.0)
    T = tail_sums(sig, n)
    for r in range(T.size):
        if math.sqrt(1.0 + r / (p - 1.0)) * math.sqrt(T[r]) <= eps * ref:
            return r
    return None


@dataclass
class QBResult:
    r: int                 # selected target rank
    k: int                 # columns of Q (r + p, or s when the criterion was not met)
    final_s: int           # sketch width at which the selection was made
    met: bool              # the criterion was met with r + p <= s
    transposed: bool
    Q: np.ndarray          # m' x k, orthonormal columns
    B: np.ndarray          # k x n'
    sigma: np.ndarray      # the trusted sketched singular values at final_s


def qb(A: np.ndarray, eps: float, p: int = 10, seed: int = 0, s0: int = 8, s_max: int = 512,
       norm_a: float | None = None) -> QBResult:
    """Algorithm 3 with the doubling of Algorithm 1 for growing the sketch."""
    if p < 2:
        raise ValueError("p must be at least 2")
    if not (0.0 < eps < 1.0):
        raise ValueError("eps must lie in (0, 1)")
    Ao, transposed = alg.orient(np.asarray(A))
    A64 = np.asarray(Ao, dtype=np.float64)
    m, n = A64.shape
    cap = alg.ladder_limits(m, n, alg.GAUSSIAN, s_max)
    s = s0
    while True:
        r1 = alg.r1_of_s(s)
        sig = alg.sketched_sigma(A64, s, alg.GAUSSIAN, seed)[:r1]
        r = select_rank(sig, n, eps, p, norm_a)
        # k = min(r + p, n) columns factor A exactly once the sketch covers all n
        # singular values: the criterion is met when those k columns are sketched
        met = r is not None and min(r + p, n) <= s
        if met or 2 * s > cap or r1 >= n:
            break
        s *= 2
    if met:
        k = min(r + p, n)
    else:
        k = min(s, n)
        r = max(k - p, 0)
    AXk = A64 @ rng.gaussian_x(n, k, seed)                 # step 6: the first k columns of AX
    Q, R = np.linalg.qr(AXk)                               # step 7
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    Q = Q * d[None, :]
    B = Q.T @ A64                                          # step 8
    return QBResult(r, k, s, met, transposed, Q, B, sig)
