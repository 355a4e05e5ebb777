"""Algorithm 1 (Sec. 5, "Rank Estimation with approximate orthogonalization") in
FP64 on the CPU.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Every step follows the algorithm box in order, with the embeddings written out
densely so that each product is a plain matrix product a reader can check:

  step 1  r~1 = round(1.1 r1)                         -> ``oversampled``
  step 2  draw X (n x r~1): Gaussian G, SRTT D H S^T, HRTT D H C^T or HRCT D F^T C^T
                                                       -> ``rng.gaussian_x`` / ``rng.srtt_x`` / ``rng.hrtt_x``
  step 3  form A X                                     -> ``A @ X``
  step 4  r2 = 2 r~1
  step 5  draw Y (r2 x m): Gaussian, SRTT S H D or S C D (C the DCT-II)
                                                       -> ``rng.gaussian_y`` / ``rng.srtt_y`` / ``rng.srct_y``
  step 6  form Y (A X)                                 -> ``Y @ AX``
  step 7  the first r1 singular values                 -> LAPACK (numpy.linalg.svd), or the
          diagonal of R in Y A X = QR as their estimates (the alternative of Sec. 5's
          remark on step 7)                            -> ``qr_diagonal_sigma``
  step 8  first r^ with sigma_{r^+1} <= eps ||A||, ||A|| ~ sigma_1(Y A X) when
          unknown; otherwise grow r1 by appending      -> ``readoff`` / ``rank_estimate``

Readings of the paper taken here (the CUDA path takes the same ones):

* Sketch width ladder.  The X width s runs over s0, 2 s0, 4 s0, ... (s0 a
  multiple of 8), r2 = 2 s, and r1(s) is the largest r1 with
  round(1.1 r1) <= s, where round() takes halves away from zero (computed as
  floor((11 r1 + 5) / 10)).  This gives s -> r1: 8->7, 16->14, 32->29, 64->58,
  128->116, 256->233, 512->465; only at s = 16 does X carry one column beyond
  round(1.1 r1) (extra oversampling).  Doubling s doubles r1 up to rounding
  ("r1 := 2 r1", step 8).
* Scaling.  X = G/sqrt(s), Y = G/sqrt(r2) (Sec. 1 notation: Gaussian embedding
  G/sqrt(r)); for the SRTT, Theta = sqrt(m_pad/r2) S (H/sqrt(m_pad)) D =
  S H D / sqrt(r2) and likewise X = D H S^T / sqrt(s).  The unscaled sketches are
  formed and sigma is multiplied by 1/sqrt(s r2) afterwards.
* Hadamard zero padding (Sec. 4): n and m are padded to the next power of two.
* HRTT (Sec. 3.4, hashed randomized transform): X = D (H/sqrt(n_pad)) C^T with
  a CountSketch C, so the singular values are scaled by 1/sqrt(n_pad r2).  Its
  columns depend on the width, so each step of the doubling loop sketches anew.
  The left embedding is Gaussian: the column space of A X is that of A's leading
  left singular vectors, coherent whenever A is (a diagonal A gives coordinate
  vectors), and a sampled Hadamard Y aliases on it as a sampled Hadamard X does
  on the right.
* m < n: the estimate is taken on A^T (Notation assumes m >= n; rank is
  invariant under transposition).
* Read-off: tau = eps * sigma^_1 (or eps * normA when the caller gives ||A||);
  r^ = min { i in [0, r1-1] : sigma^_{i+1} <= tau } (only the first r1 values
  are trusted, Sec. 3.3); "<=" as in Definition 1.  If no such i exists the
  sketch is grown; when it cannot grow, r1 is returned as a lower bound (Sec. 5).
* Gap measure (step 8, last sentence, printed garbled as a max): the index
  g = argmax_{1<=i<r1} sigma^_i / sigma^_{i+1}, smallest i on ties, with the ratio
  +inf when sigma^_{i+1} = 0 < sigma^_i and 1 when both are 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import rng

GAUSSIAN = 0
SRHT = 1
HRTT = 2
SRCT = 3        # left embedding only: subsampled randomized DCT (Sec. 4, eta = 2)
HRCT = 4        # right embedding only: hashed randomized DCT (Sec. 3.4, the experiments' X)


def round_half_away(num: int, den: int) -> int:
    """round(num/den) with halves away from zero, for num, den >= 0 integers."""
    return (2 * num + den) // (2 * den)


def oversampled(r1: int) -> int:
    """Step 1: r~1 = round(1.1 r1)."""
    return round_half_away(11 * r1, 10)


def r1_of_s(s: int) -> int:
    """Largest r1 >= 1 whose oversampled width round(1.1 r1) fits in s columns."""
    r = 1
    while oversampled(r + 1) <= s:
        r += 1
    return r


def embeddings(kind: int, n: int, m: int, s: int, seed: int,
               col0: int = 0, row0: int = 0, r2: int | None = None):
    """Steps 2 and 5: unscaled X[:, col0:col0+s] (n x s) and Y[row0:row0+r2, :]."""
    r2 = 2 * s if r2 is None else r2
    if kind == GAUSSIAN:
        return rng.gaussian_x(n, s, seed, col0), rng.gaussian_y(r2, m, seed, row0)
    if kind == SRHT:
        return rng.srtt_x(n, s, seed, col0), rng.srtt_y(r2, m, seed, row0)
    if kind in (HRTT, HRCT):
        if col0 != 0:
            raise ValueError("hashed embeddings' columns depend on the width: col0 must be 0")
        X = rng.hrtt_x(n, s, seed) if kind == HRTT else rng.hrct_x(n, s, seed)
        return X, rng.gaussian_y(r2, m, seed, row0)
    raise ValueError(f"unknown sketch kind {kind}")


def left_kind(kind: int) -> int:
    """Kind of the left embedding Y drawn with right embedding `kind`."""
    return GAUSSIAN if kind in (HRTT, HRCT) else kind


def orient(A: np.ndarray) -> tuple[np.ndarray, bool]:
    """A as an m' x n' matrix with m' >= n' (transposed when m < n)."""
    A = np.asarray(A)
    if A.shape[0] < A.shape[1]:
        return A.T, True
    return A, False


def right_sketch(A: np.ndarray, s: int, kind: int, seed: int, col0: int = 0) -> np.ndarray:
    """Steps 2-3: A X for columns col0..col0+s-1 of the unscaled embedding."""
    A64 = np.asarray(A, dtype=np.float64)
    X = embeddings(kind, A64.shape[1], A64.shape[0], s, seed, col0=col0, r2=0)[0]
    return A64 @ X


def left_sketch(AX: np.ndarray, r2: int, kind: int, seed: int, row0: int = 0, ykind: int | None = None) -> np.ndarray:
    """Steps 5-6: Y (A X) for rows row0..row0+r2-1 of the unscaled embedding (Y of
    kind `ykind`, by default the one drawn with right embedding `kind`)."""
    m = AX.shape[0]
    yk = left_kind(kind) if ykind is None else ykind
    if yk == GAUSSIAN:
        Y = rng.gaussian_y(r2, m, seed, row0)
    elif yk == SRHT:
        Y = rng.srtt_y(r2, m, seed, row0)
    elif yk == SRCT:
        Y = rng.srct_y(r2, m, seed, row0)
    else:
        raise ValueError(f"unknown left embedding {yk}")
    return Y @ AX


def sketch_scale(s: int, kind: int = GAUSSIAN, n: int = 0) -> float:
    """1/sqrt(s * r2) with r2 = 2 s; for the hashed embeddings 1/sqrt(n_pad * r2) (n columns)."""
    if kind in (HRTT, HRCT):
        return 1.0 / math.sqrt(float(1 << rng.next_pow2_bits(n)) * float(2 * s))
    return 1.0 / math.sqrt(float(s) * float(2 * s))


def core(A: np.ndarray, s: int, kind: int, seed: int, ykind: int | None = None) -> np.ndarray:
    """Unscaled 2s x s core Y A X of an already oriented (m >= n) matrix."""
    AX = right_sketch(A, s, kind, seed)
    return left_sketch(AX, 2 * s, kind, seed, ykind=ykind)


def qr_diagonal_sigma(C: np.ndarray) -> np.ndarray:
    """Step 7 by the remark after Algorithm 1 (Sec. 5): factor the core C = QR
    (Householder, LAPACK) and take |R_kk| as estimates of sigma_k(C) -- a QR of a
    matrix whose right singular vectors are randomised reveals its rank with high
    probability.  Reading: the estimates are sorted descending, so that the
    read-off's "first r^" and sigma^_1 (the largest estimate, for ||A||) are taken
    on an ordered list as with singular values."""
    R = np.linalg.qr(np.asarray(C, dtype=np.float64), mode="r")
    return np.sort(np.abs(np.diag(R)))[::-1]


def sketched_sigma(A: np.ndarray, s: int, kind: int, seed: int, sigma: str = "svd",
                   ykind: int | None = None) -> np.ndarray:
    """Step 7: all s singular values of Y A X (or their QR-diagonal estimates),
    scaled (descending, FP64)."""
    C = core(A, s, kind, seed, ykind)
    sig = np.linalg.svd(C, compute_uv=False) if sigma == "svd" else qr_diagonal_sigma(C)
    return sig * sketch_scale(s, kind, np.shape(A)[1])


@dataclass
class Readoff:
    rank: int | None          # None when no sigma^_{i+1} <= tau among the trusted values
    gap_index: int
    gap_ratio: float
    tau: float


def readoff(sig_trusted: np.ndarray, eps: float, norm_a: float | None = None) -> Readoff:
    """Step 8 on the first r1 sketched singular values."""
    sig = np.asarray(sig_trusted, dtype=np.float64)
    r1 = sig.shape[0]
    ref = norm_a if (norm_a is not None and norm_a > 0) else sig[0]
    tau = eps * ref
    rank = None
    for i in range(r1):               # r^ = i means sigma^_{i+1} <= tau (1-based)
        if sig[i] <= tau:
            rank = i
            break
    gi, gr = 1, -1.0
    for i in range(1, r1):            # ratio sigma^_i / sigma^_{i+1}, 1-based i
        a, b = sig[i - 1], sig[i]
        if b > 0:
            ratio = a / b
        elif a > 0:
            ratio = math.inf
        else:
            ratio = 1.0
        if ratio > gr:
            gi, gr = i, ratio
    if r1 < 2:
        gi, gr = 1 if r1 == 1 else 0, 1.0
    return Readoff(rank, gi, gr, tau)


@dataclass
class Result:
    rank: int
    converged: bool
    transposed: bool
    final_s: int
    passes: int
    sigma: np.ndarray                 # first r1(final_s) scaled sketched singular values
    gap_index: int
    gap_ratio: float
    history: list = field(default_factory=list)   # (s, r1, rank or None) per step


def ladder_limits(m: int, n: int, kind: int, s_max: int, ykind: int | None = None) -> int:
    """Largest admissible sketch width for an oriented m x n matrix (m >= n)."""
    cap = s_max
    yk = left_kind(kind) if ykind is None else ykind
    if kind == SRHT:
        cap = min(cap, 1 << rng.next_pow2_bits(n))
    if yk in (SRHT, SRCT):
        cap = min(cap, (1 << rng.next_pow2_bits(m)) // 2)   # 2s sampled rows of the padded transform
    if kind in (HRTT, HRCT):
        cap = min(cap, 1 << rng.next_pow2_bits(n))      # no empty bucket
    return cap


def rank_estimate(A: np.ndarray, eps: float, kind: int = GAUSSIAN, seed: int = 0,
                  s0: int = 8, s_max: int = 512, norm_a: float | None = None, sigma: str = "svd",
                  ykind: int | None = None) -> Result:
    """Algorithm 1 with the doubling loop of step 8 (appending to X and Y).

    Each step recomputes the core from the plain definition Y[:2s] A X[:, :s];
    for the Gaussian and SRTT embeddings column j of X and row q of Y do not
    depend on s, so this is the same matrix the appended sketches give (the
    HRTT's X does depend on s and is drawn anew at every step).
    """
    A = np.asarray(A)
    if A.ndim != 2:
        raise ValueError("A must be 2-D")
    if not (0.0 < eps < 1.0):
        raise ValueError("eps must lie in (0, 1)")
    if s0 < 8 or s0 % 8 != 0 or s_max < s0:
        raise ValueError("s0 must be a positive multiple of 8 and s_max >= s0")
    if not np.all(np.isfinite(A)):
        raise ValueError("A has non-finite entries")
    Ao, transposed = orient(A)
    m, n = Ao.shape
    if m == 0 or n == 0:
        raise ValueError("empty matrix")
    cap = ladder_limits(m, n, kind, s_max, ykind)
    if s0 > cap:
        raise ValueError("initial sketch width exceeds the admissible width")
    A64 = np.asarray(Ao, dtype=np.float64)
    s = s0
    history = []
    passes = 0
    while True:
        passes += 1
        sig_all = sketched_sigma(A64, s, kind, seed, sigma, ykind)
        r1 = r1_of_s(s)
        sig = sig_all[:r1]
        ro = readoff(sig, eps, norm_a)
        history.append((s, r1, ro.rank))
        if ro.rank is not None:
            return Result(ro.rank, True, transposed, s, passes, sig, ro.gap_index,
                          ro.gap_ratio, history)
        if 2 * s > cap or r1 >= n:
            return Result(r1, False, transposed, s, passes, sig, ro.gap_index,
                          ro.gap_ratio, history)
        s *= 2


def numerical_rank(sigma: np.ndarray, eps: float) -> int:
    """Definition 1: the relative eps-rank from exact singular values (descending)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.size == 0:
        return 0
    tau = eps * sigma[0]
    for i in range(sigma.size):
        if sigma[i] <= tau:
            return i
    return sigma.size
