"""Counter-based random embeddings for the oracle (test infrastructure only).

The rank estimator draws a Gaussian or SRTT right embedding X (n x s) and a
Gaussian or SRTT left embedding Y (r2 x m) (Sec. 1 notation; Eq. (Theta) in
Sec. 4; Algorithm 1 steps 2 and 5).  Both sides of the parity check must draw the
*same* X and Y, so each side implements one counter-based generator from its
published definition; this module is the CPU implementation and shares no code
with the CUDA implementation.

Specification (the CUDA side follows the same text):

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): counter (c0,c1,c2,c3), key (k0,k1) = (seed mod 2^32,
  seed >> 32).  One round: (hi0,lo0) = mulhilo(0xD2511F53, c0),
  (hi1,lo1) = mulhilo(0xCD9E8D57, c2), c <- (hi1^c1^k0, lo1, hi0^c3^k1, lo0);
  the key is bumped by (0x9E3779B9, 0xBB67AE85) between rounds; 10 rounds.
* Normal transform (Box & Muller 1958) in IEEE binary32 with every operation
  correctly rounded and no fused multiply-add, using a project-written natural
  logarithm (the atanh series ln f = 2 atanh((f-1)/(f+1)) after reducing f to
  [sqrt(1/2), sqrt(2))) and project-written sine/cosine (Taylor polynomials on a
  quarter period).  Two 32-bit words give two normals; the result is rounded to
  BF16 (round to nearest even) and then to the nearest multiple of 2^-13 (ties to
  even, zero as +0).  Values of magnitude >= 2^-6 are BF16 multiples of 2^-13
  already, so the second rounding moves only smaller values, by at most 2^-14.
  Every entry is then an integer multiple of 2^-13 below 6 in magnitude (a
  16-bit fixed-point number), exact in BF16, FP16, FP32 and FP64.
* Gaussian X (n x s, unscaled G): entry (k, j) is normal t = j mod 4 of
  Philox((k, j div 4, STREAM_GX, 0)).  Gaussian Y (r2 x m, unscaled G): entry
  (q, i) is normal t = q mod 4 of Philox((i, q div 4, STREAM_GY, 0)).  Column j of
  X and row q of Y never depend on s, so growing the sketch appends (Sec. 5,
  "appending to the sketches").
* SRTT signs D: d_j = 1 - 2*bit(j mod 128) of Philox((j div 128, 0, stream, 0))
  (bit b of the 128-bit output = bit (b mod 32) of word b div 32).
* SRTT sampling S without replacement (App. A, Lemma 9 samples "without
  replacement"): the sampled index k is pi(k), pi a 4-round keyed Feistel
  bijection of [0, 2^b) whose round function is word 0 of
  Philox((half, round, stream, 0)).
* HRTT hashing (Sec. 3.4: the sampling S replaced by a CountSketch hashing
  matrix C, s x n_pad, one nonzero per column): coordinate c of the transform
  goes to bucket h(c) = pi_X^{-1}(c) mod s with sign sigma_c (a sign of stream
  SX, drawn like d_j), so bucket k holds {pi_X(k + t s) : k + t s < n_pad}.  D
  and pi are the SRTT's (streams DX and PX).

Stream identifiers: GX=1, GY=2, DX=3, PX=4, DY=5, PY=6, SX=7.
"""
from __future__ import annotations

import math

import numpy as np

STREAM_GX = 1
STREAM_GY = 2
STREAM_DX = 3
STREAM_PX = 4
STREAM_DY = 5
STREAM_PY = 6
STREAM_SX = 7

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def split_seed(seed: int) -> tuple[int, int]:
    """Philox key (k0, k1) for a 64-bit seed."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32 with 10 rounds on arrays of counters (broadcast), scalar key.

    Returns four uint32 arrays.  Written from the SC'11 definition.
    """
    c0, c1, c2, c3 = np.broadcast_arrays(
        np.asarray(c0, dtype=np.uint64), np.asarray(c1, dtype=np.uint64),
        np.asarray(c2, dtype=np.uint64), np.asarray(c3, dtype=np.uint64))
    x0 = c0 & _MASK32
    x1 = c1 & _MASK32
    x2 = c2 & _MASK32
    x3 = c3 & _MASK32
    key0 = int(k0) & 0xFFFFFFFF
    key1 = int(k1) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            key0 = (key0 + _W0) & 0xFFFFFFFF
            key1 = (key1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * x0
        p1 = _M1 * x2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x0, x1, x2, x3 = (hi1 ^ x1 ^ np.uint64(key0), lo1,
                          hi0 ^ x3 ^ np.uint64(key1), lo0)
    return (x0.astype(np.uint32), x1.astype(np.uint32),
            x2.astype(np.uint32), x3.astype(np.uint32))


# ---------------------------------------------------------------------------
# binary32 constants (exact values written as hexadecimal floats)
_f = np.float32
_C_INV = [_f(float.fromhex(h)) for h in (
    "0x1.555556p-2", "0x1.99999ap-3", "0x1.24924ap-3", "0x1.c71c72p-4",
    "0x1.745d18p-4")]                      # 1/3, 1/5, 1/7, 1/9, 1/11
_LN2 = _f(float.fromhex("0x1.62e430p-1"))
_SQRT2 = _f(float.fromhex("0x1.6a09e6p+0"))
_HALF_PI = _f(float.fromhex("0x1.921fb6p+0"))
_SIN_C = [_f(float.fromhex(h)) for h in (   # (-1)^k / (2k+1)!, k = 1..6
    "-0x1.555556p-3", "0x1.111112p-7", "-0x1.a01a02p-13", "0x1.71de3ap-19",
    "-0x1.ae6456p-26", "0x1.612462p-33")]
_COS_C = [_f(float.fromhex(h)) for h in (   # (-1)^k / (2k)!, k = 1..7
    "-0x1.000000p-1", "0x1.555556p-5", "-0x1.6c16c2p-10", "0x1.a01a02p-16",
    "-0x1.27e4fcp-22", "0x1.1eed8ep-29", "-0x1.93974ap-37")]
_TWO_M24 = _f(2.0 ** -24)
_ONE = _f(1.0)
_TWO = _f(2.0)
_HALF = _f(0.5)
_FOUR = _f(4.0)


def ln_f32(u: np.ndarray) -> np.ndarray:
    """Natural log of positive normal binary32 values, binary32 arithmetic.

    u = f * 2^e with f in [1, 2) taken from the bit pattern; f is halved when
    above sqrt(2); then ln u = e ln2 + 2 t (1 + t^2/3 + ... + t^10/11) with
    t = (f-1)/(f+1), |t| <= 0.172 (atanh series, truncation < 1e-10).
    """
    u = np.asarray(u, dtype=np.float32)
    bits = u.view(np.uint32)
    e = ((bits >> np.uint32(23)) & np.uint32(0xFF)).astype(np.int32) - 127
    fbits = (bits & np.uint32(0x007FFFFF)) | np.uint32(0x3F800000)
    f = fbits.view(np.float32).copy()
    big = f > _SQRT2
    f = np.where(big, f * _HALF, f).astype(np.float32)
    e = np.where(big, e + 1, e)
    t = ((f - _ONE) / (f + _ONE)).astype(np.float32)
    t2 = (t * t).astype(np.float32)
    p = _C_INV[4]
    for c in (_C_INV[3], _C_INV[2], _C_INV[1], _C_INV[0]):
        p = (p * t2 + c).astype(np.float32)          # two roundings (no fma)
    p = (p * t2 + _ONE).astype(np.float32)
    lnf = ((_TWO * t).astype(np.float32) * p).astype(np.float32)
    return (e.astype(np.float32) * _LN2 + lnf).astype(np.float32)


def sincos_quarter_f32(theta: np.ndarray):
    """sin and cos of theta in [0, pi/2) by Horner-evaluated Taylor polynomials."""
    th = np.asarray(theta, dtype=np.float32)
    t2 = (th * th).astype(np.float32)
    ps = _SIN_C[5]
    for c in (_SIN_C[4], _SIN_C[3], _SIN_C[2], _SIN_C[1], _SIN_C[0]):
        ps = (ps * t2 + c).astype(np.float32)
    ps = (ps * t2).astype(np.float32)
    s = (th * ps + th).astype(np.float32)            # th + th^3 (...)
    pc = _COS_C[6]
    for c in (_COS_C[5], _COS_C[4], _COS_C[3], _COS_C[2], _COS_C[1], _COS_C[0]):
        pc = (pc * t2 + c).astype(np.float32)
    c_ = (pc * t2 + _ONE).astype(np.float32)
    return s, c_


def round_bf16(z: np.ndarray) -> np.ndarray:
    """Round binary32 to the nearest BF16 (ties to even), as binary32."""
    z = np.asarray(z, dtype=np.float32)
    bits = z.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    bits = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return bits.view(np.float32).copy()


def round_normal(z: np.ndarray) -> np.ndarray:
    """Round binary32 to BF16 (ties to even), then to the nearest multiple of
    2^-13 (ties to even; zero as +0)."""
    r = round_bf16(z)
    t = (np.round(r.astype(np.float64) * 8192.0) / 8192.0).astype(np.float32)   # numpy rounds ties to even
    r = np.where(np.abs(r) < _f(2.0 ** -6), t, r).astype(np.float32)
    r[r == 0] = _f(0.0)
    return r


def box_muller_bf16(a: np.ndarray, b: np.ndarray):
    """Two standard normals (BF16-exact multiples of 2^-13) from two uint32 words (Box-Muller)."""
    a = np.asarray(a, dtype=np.uint32)
    b = np.asarray(b, dtype=np.uint32)
    u1 = ((a >> np.uint32(8)).astype(np.float32) + _ONE) * _TWO_M24     # (0, 1]
    u2 = (b >> np.uint32(8)).astype(np.float32) * _TWO_M24              # [0, 1)
    u1 = u1.astype(np.float32)
    u2 = u2.astype(np.float32)
    w = (_f(-2.0) * ln_f32(u1)).astype(np.float32)
    r = np.sqrt(w).astype(np.float32)
    v = (u2 * _FOUR).astype(np.float32)
    q = np.floor(v).astype(np.int32)
    fr = (v - q.astype(np.float32)).astype(np.float32)
    theta = (fr * _HALF_PI).astype(np.float32)
    s, c = sincos_quarter_f32(theta)
    cos_phi = np.select([q == 0, q == 1, q == 2], [c, -s, -c], s).astype(np.float32)
    sin_phi = np.select([q == 0, q == 1, q == 2], [s, c, -s], -c).astype(np.float32)
    z0 = (r * cos_phi).astype(np.float32)
    z1 = (r * sin_phi).astype(np.float32)
    return round_normal(z0), round_normal(z1)


def normals4(c0, c1, stream: int, seed: int):
    """The four normals of Philox((c0, c1, stream, 0)) as float32 arrays."""
    k0, k1 = split_seed(seed)
    x0, x1, x2, x3 = philox4x32_10(c0, c1, stream, 0, k0, k1)
    z0, z1 = box_muller_bf16(x0, x1)
    z2, z3 = box_muller_bf16(x2, x3)
    return z0, z1, z2, z3


def gaussian_x(n: int, s: int, seed: int, col0: int = 0) -> np.ndarray:
    """Unscaled Gaussian right embedding G[:, col0:col0+s] (n x s), float64."""
    if n == 0 or s == 0:
        return np.empty((n, s), dtype=np.float64)
    g0, g1 = col0 // 4, (col0 + s + 3) // 4
    k = np.arange(n, dtype=np.int64)[:, None]
    g = np.arange(g0, g1, dtype=np.int64)[None, :]
    z = normals4(k, g, STREAM_GX, seed)                    # four (n, groups)
    full = np.stack(z, axis=2).reshape(n, 4 * (g1 - g0))    # column 4g+t
    off = col0 - 4 * g0
    return full[:, off:off + s].astype(np.float64)


def gaussian_y(r2: int, m: int, seed: int, row0: int = 0) -> np.ndarray:
    """Unscaled Gaussian left embedding G[row0:row0+r2, :] (r2 x m), float64."""
    if r2 == 0 or m == 0:
        return np.empty((r2, m), dtype=np.float64)
    g0, g1 = row0 // 4, (row0 + r2 + 3) // 4
    i = np.arange(m, dtype=np.int64)[None, :]
    g = np.arange(g0, g1, dtype=np.int64)[:, None]
    z = normals4(i, g, STREAM_GY, seed)                    # four (groups, m)
    full = np.stack(z, axis=1).reshape(4 * (g1 - g0), m)    # row 4g+t
    off = row0 - 4 * g0
    return full[off:off + r2, :].astype(np.float64)


def signs(count: int, stream: int, seed: int) -> np.ndarray:
    """Random signs d_0..d_{count-1} in {+1, -1} (the diagonal D of Eq. (Theta))."""
    if count == 0:
        return np.empty(0, dtype=np.float64)
    k0, k1 = split_seed(seed)
    j = np.arange(count, dtype=np.int64)
    words = philox4x32_10(j // 128, 0, stream, 0, k0, k1)
    w = np.stack(words, axis=0).astype(np.uint64)            # 4 x count
    widx = (j % 128) // 32
    bit = (j % 32).astype(np.uint64)
    chosen = w[widx, np.arange(count)]
    b = (chosen >> bit) & np.uint64(1)
    return 1.0 - 2.0 * b.astype(np.float64)


def feistel_perm(x, bits: int, stream: int, seed: int) -> np.ndarray:
    """4-round keyed Feistel bijection of [0, 2^bits) evaluated at x."""
    x = np.asarray(x, dtype=np.int64)
    if bits == 0:
        return np.zeros_like(x)
    k0, k1 = split_seed(seed)
    w_lo = bits // 2
    w_hi = bits - w_lo
    lo = x & ((1 << w_lo) - 1)
    hi = x >> w_lo
    for rnd in range(4):
        f = philox4x32_10(hi, rnd, stream, 0, k0, k1)[0].astype(np.int64)
        new_lo = hi
        new_hi = lo ^ (f & ((1 << w_lo) - 1))
        lo, hi = new_lo, new_hi
        w_lo, w_hi = w_hi, w_lo
    return (hi << w_lo) | lo


def next_pow2_bits(n: int) -> int:
    """b with 2^b the smallest power of two >= n (the zero padding of Sec. 4)."""
    b = 0
    while (1 << b) < n:
        b += 1
    return b


_PARITY16 = None


def _parity16() -> np.ndarray:
    """parity(popcount(v)) for every 16-bit v, by shifting out the bits."""
    global _PARITY16
    if _PARITY16 is None:
        a = np.arange(1 << 16, dtype=np.int64)
        par = np.zeros_like(a)
        while np.any(a):
            par ^= a & 1
            a = a >> 1
        _PARITY16 = par.astype(np.uint8)
    return _PARITY16


def hadamard_entries(rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
    """Sylvester Hadamard entries H[i, c] = (-1)^popcount(i & c), float64
    (indices below 2^32; the parity of i & c from its two 16-bit halves)."""
    a = np.bitwise_and(np.asarray(rows, dtype=np.int64)[:, None],
                       np.asarray(cols, dtype=np.int64)[None, :])
    if a.size and int(a.max()) >> 32:
        raise ValueError("Hadamard index beyond 2^32")
    t = _parity16()
    par = t[a & 0xFFFF] ^ t[a >> 16]
    return 1.0 - 2.0 * par.astype(np.float64)


def srtt_x(n: int, s: int, seed: int, col0: int = 0) -> np.ndarray:
    """Unscaled subsampled randomized Hadamard right embedding, n x s.

    X = D H S^T over the zero-padded dimension n_pad = 2^ceil(log2 n) (Eq. (Theta)
    transposed; Sec. 4 on zero padding for the Hadamard transform); column j
    samples Hadamard column pi_X(j).  The scale 1/sqrt(s) is applied to the
    singular values afterwards.
    """
    b = next_pow2_bits(n)
    d = signs(n, STREAM_DX, seed)
    cols = feistel_perm(np.arange(col0, col0 + s), b, STREAM_PX, seed)
    return d[:, None] * hadamard_entries(np.arange(n), cols)


def srtt_y(r2: int, m: int, seed: int, row0: int = 0) -> np.ndarray:
    """Unscaled subsampled randomized Hadamard left embedding, r2 x m (Eq. (Theta))."""
    b = next_pow2_bits(m)
    d = signs(m, STREAM_DY, seed)
    rows = feistel_perm(np.arange(row0, row0 + r2), b, STREAM_PY, seed)
    return hadamard_entries(rows, np.arange(m)) * d[None, :]


def hrct_x(n: int, s: int, seed: int, rows=None) -> np.ndarray:
    """Unscaled hashed randomized DCT right embedding, n x s: X = D F^T C^T with F
    the DCT-II of order n_pad = 2^ceil(log2 n) scaled to entries of magnitude up to
    sqrt(2) (sqrt(n_pad) times the orthonormal transform) and C the CountSketch of
    hrtt_x (the same buckets {pi(k + t s)} and signs sigma_c) -- the hashed
    randomized DCT the paper's experiments use for X (Sec. 3.4, Sec. 6).  Column k
    of X is d * sum over its bucket of sigma_c F[c, :].  The orthonormal
    transform's scale 1/sqrt(n_pad) is applied to the singular values afterwards."""
    if s < 1:
        raise ValueError("s must be positive")
    b = next_pow2_bits(n)
    n_pad = 1 << b
    if s > n_pad:
        raise ValueError("HRCT width exceeds the padded dimension (empty buckets)")
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    d = signs(n, STREAM_DX, seed)[rows]
    sigma = signs(n_pad, STREAM_SX, seed)
    X = np.empty((rows.size, s), dtype=np.float64)
    for k in range(s):
        c = feistel_perm(np.arange(k, n_pad, s), b, STREAM_PX, seed)   # bucket k
        X[:, k] = d * (dct_entries(c, rows, n_pad).T @ sigma[c])
    return X


def dct_entries(rows: np.ndarray, cols: np.ndarray, N: int) -> np.ndarray:
    """sqrt(N) times the orthonormal DCT-II matrix of order N, rows k x columns i:
    sqrt(2) w_k cos(pi (2 i + 1) k / (2 N)), w_0 = 1/sqrt(2), w_k = 1 otherwise.
    The phase (2 i + 1) k is reduced modulo 4 N in integers before the cosine."""
    k = np.asarray(rows, dtype=np.int64)[:, None]
    i = np.asarray(cols, dtype=np.int64)[None, :]
    ph = ((2 * i + 1) * k) % (4 * N)
    v = math.sqrt(2.0) * np.cos(np.pi * ph.astype(np.float64) / (2.0 * N))
    return np.where(k == 0, 1.0, v)


def srct_y(r2: int, m: int, seed: int, row0: int = 0) -> np.ndarray:
    """Unscaled subsampled randomized DCT left embedding, r2 x m (Eq. (Theta) with F
    the orthonormal DCT-II, coherence eta = 2: the transform the paper's
    experiments use for Y, Sec. 4 and Sec. 6).  As for the Hadamard form the order
    is the zero-padded m_pad = 2^ceil(log2 m), row q samples frequency pi_Y(q)
    (stream PY) and D holds the signs of stream DY; the entries are
    sqrt(m_pad) F D, so Theta = Y / sqrt(r2)."""
    b = next_pow2_bits(m)
    d = signs(m, STREAM_DY, seed)
    rows = feistel_perm(np.arange(row0, row0 + r2), b, STREAM_PY, seed)
    return dct_entries(rows, np.arange(m), 1 << b) * d[None, :]


def hrtt_x(n: int, s: int, seed: int, rows=None) -> np.ndarray:
    """Unscaled hashed randomized Hadamard right embedding, n x s: X = D H C^T
    (only the given rows when `rows` is not None).

    Sec. 3.4 (HRTT): Eq. (Theta) with the sampling matrix S replaced by a
    hashing matrix; here C[h(c), c] = sigma_c with h(c) = pi^{-1}(c) mod s over
    the zero-padded dimension n_pad = 2^ceil(log2 n).  Column k of X is
    d * sum over the bucket {c = pi(k + t s)} of sigma_c H[:, c].  The columns
    depend on s (the width is not appendable).  The orthonormal transform's
    scale 1/sqrt(n_pad) is applied to the singular values afterwards.
    """
    if s < 1:
        raise ValueError("s must be positive")
    b = next_pow2_bits(n)
    n_pad = 1 << b
    if s > n_pad:
        raise ValueError("HRTT width exceeds the padded dimension (empty buckets)")
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    d = signs(n, STREAM_DX, seed)[rows]
    sigma = signs(n_pad, STREAM_SX, seed)
    X = np.empty((rows.size, s), dtype=np.float64)
    for k in range(s):
        c = feistel_perm(np.arange(k, n_pad, s), b, STREAM_PX, seed)   # bucket k
        X[:, k] = d * (hadamard_entries(rows, c) @ sigma[c])
    return X
