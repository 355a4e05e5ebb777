"""Seeded synthetic test matrices with prescribed singular values.

This module only builds inputs; it holds none of the rank estimator's
arithmetic.  Both the CUDA path's tests/benchmark and the CPU oracle draw their
matrices from here.  The spectra follow the paper's synthetic families (Sec. 6:
step gaps A_G, polynomial decay A_SP/A_FP, exponential decay A_SE/A_FE) and the
workloads the rank estimator is measured on:

* ``haar_matrix``: A = U diag(sigma) V^T with U (m x n) and V (n x n) the Q
  factors of QR of seeded N(0,1) matrices (column signs fixed by diag(R) > 0);
  used for the 2048 x 1024 FP64 case with sigma_i = 10^{-(i-1)/10} (i <= 60),
  then 1e-12.
* ``householder_matrix``: U = H_1..H_8 D_u, V = H'_1..H'_8 D_v with H = I - 2 v v^T
  for seeded unit Gaussian v and random sign diagonals D; cheap enough to build
  65536 x 16384 on the device (sigma_i = 1 for i <= 200, then 1e-6 / i).
* ``kernel_blocks``: K_ij = 1 / |x_i - y_j| for x uniform in [0,1]^3 and y uniform
  in a unit box shifted by 1 + d along the first axis, d ~ U[1, 4]; block sizes
  m, n ~ U{256..4096} (off-diagonal blocks of a hierarchical matrix, Sec. 1).
"""
from __future__ import annotations

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


# ---------------------------------------------------------------------------
# spectra
def spectrum(family: str, n: int, *, rank: int = 40, **kw) -> torch.Tensor:
    """Singular values (descending, FP64) of a named synthetic family.

    gaps:  1 (i<=100), 1e-4 (<=200), 1e-8 (<=300), 1e-12 (<=400), 1e-16 after
           (the block length 100 can be changed with ``block``).
    sp/fp: i^-1 and i^-3.        se/fe: 10^{-0.01 (i-1)} and 10^{-0.5 (i-1)}.
    decade10: 10^{-(i-1)/10} for i <= ``head`` (60), then ``floor`` (1e-12).
    step:  1 for i <= ``rank``, then ``tail_scale`` / i (default 1e-6 / i).
    geom300: 10^{-10 (i-1)/300} for i <= 300, then ``floor`` (1e-12).
    """
    i = torch.arange(1, n + 1, dtype=torch.float64)
    if family == "gaps":
        b = kw.get("block", 100)
        lev = torch.clamp((i - 1) // b, max=4)
        return torch.pow(10.0, -4.0 * lev)
    if family == "sp":
        return 1.0 / i
    if family == "fp":
        return i ** -3.0
    if family == "se":
        return torch.pow(10.0, -0.01 * (i - 1))
    if family == "fe":
        return torch.pow(10.0, -0.5 * (i - 1))
    if family == "decade10":
        head = kw.get("head", 60)
        floor = kw.get("floor", 1e-12)
        s = torch.pow(10.0, -(i - 1) / 10.0)
        s[head:] = floor
        return s
    if family == "step":
        tail = kw.get("tail_scale", 1e-6)
        s = tail / i
        s[:rank] = 1.0
        return s
    if family == "geom300":
        floor = kw.get("floor", 1e-12)
        s = torch.pow(10.0, -10.0 * (i - 1) / 300.0)
        s[300:] = floor
        return s
    raise ValueError(f"unknown spectrum family {family!r}")


# ---------------------------------------------------------------------------
# dense matrices with a prescribed spectrum
def haar_orthonormal(m: int, k: int, seed: int, device="cpu") -> torch.Tensor:
    """m x k matrix with orthonormal columns, Haar distributed (QR of N(0,1))."""
    g = _gen(seed, device)
    G = torch.randn(m, k, generator=g, dtype=torch.float64, device=device)
    # the factorisation runs on the host (the device linear-algebra library is an
    # optional part of PyTorch installs; the input numbers stay the device draw)
    Q, R = torch.linalg.qr(G.cpu())
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return (Q * d).to(device)


def haar_matrix(m: int, n: int, sigma: torch.Tensor, seed: int, device="cpu",
                dtype=torch.float64) -> torch.Tensor:
    """A = U diag(sigma) V^T with Haar U (m x k), V (n x k), k = len(sigma) <= min(m, n)."""
    k = sigma.numel()
    U = haar_orthonormal(m, k, 2 * seed + 1, device)
    V = haar_orthonormal(n, k, 2 * seed + 2, device)
    A = (U * sigma.to(device)) @ V.T
    return A.to(dtype).contiguous()


def _reflect_left(C: torch.Tensor, v: torch.Tensor) -> None:
    """C <- (I - 2 v v^T) C in place."""
    w = v @ C
    C.sub_(2.0 * torch.outer(v, w))


def _reflect_right(B: torch.Tensor, v: torch.Tensor) -> None:
    """B <- B (I - 2 v v^T) in place."""
    w = B @ v
    B.sub_(2.0 * torch.outer(w, v))


def householder_matrix(m: int, n: int, sigma: torch.Tensor, seed: int, device="cpu",
                       dtype=torch.float32, reflectors: int = 8) -> torch.Tensor:
    """A = U[:, :n] diag(sigma) V^T, U = H_1..H_8 D_u (m x m), V = H'_1..H'_8 D_v (n x n).

    ``sigma`` has n entries (m >= n).  Built in FP64 on ``device``, then cast.
    """
    assert m >= n and sigma.numel() == n
    g = _gen(seed, device)
    du = torch.randint(0, 2, (n,), generator=g, device=device).to(torch.float64) * 2 - 1
    dv = torch.randint(0, 2, (n,), generator=g, device=device).to(torch.float64) * 2 - 1
    vs_u = [torch.randn(m, generator=g, dtype=torch.float64, device=device) for _ in range(reflectors)]
    vs_v = [torch.randn(n, generator=g, dtype=torch.float64, device=device) for _ in range(reflectors)]
    vs_u = [v / torch.linalg.vector_norm(v) for v in vs_u]
    vs_v = [v / torch.linalg.vector_norm(v) for v in vs_v]
    # B = diag(sigma) V^T = diag(sigma) D_v H'_8 ... H'_1
    B = torch.diag(sigma.to(device)) * dv[None, :]
    for v in reversed(vs_v):
        _reflect_right(B, v)
    # A = H_1 ... H_8 [D_u[:n] B; 0]
    C = torch.zeros(m, n, dtype=torch.float64, device=device)
    C[:n] = du[:, None] * B
    del B
    for v in reversed(vs_u):
        _reflect_left(C, v)
    return C.to(dtype).contiguous()


def kernel_points(m: int, n: int, seed: int, device="cpu"):
    """Point sets of a kernel block (FP64): x ~ U[0,1]^3 (m points) and
    y ~ U[0,1]^3 + (1 + d) e_1 (n points), d ~ U[1, 4]."""
    g = _gen(seed, device)
    d = 1.0 + 3.0 * torch.rand((), generator=g, dtype=torch.float64, device=device)
    x = torch.rand(m, 3, generator=g, dtype=torch.float64, device=device)
    y = torch.rand(n, 3, generator=g, dtype=torch.float64, device=device)
    y[:, 0] += 1.0 + d
    return x, y


def kernel_block(m: int, n: int, seed: int, device="cpu", dtype=torch.float32) -> torch.Tensor:
    """K_ij = 1/|x_i - y_j| for the points of kernel_points."""
    x, y = kernel_points(m, n, seed, device)
    K = 1.0 / torch.cdist(x, y)
    return K.to(dtype).contiguous()


def kernel_block_sizes(count: int, seed: int, lo: int = 256, hi: int = 4096):
    """Seeded block shapes (m, n), each uniform on {lo..hi}."""
    g = _gen(seed, "cpu")
    mn = torch.randint(lo, hi + 1, (count, 2), generator=g)
    return [(int(a), int(b)) for a, b in mn.tolist()]
