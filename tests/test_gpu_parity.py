"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: integer and index results bit-exact (generator outputs, sampled Hadamard
columns, ranks on inputs with a clear gap); floating point within tolerances
derived from FP32 arithmetic (stated per test); sketched singular values within
1e-4 * sigma^_1 of the oracle's.
"""
import math

import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from oracle import rng
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

from rankcheck import decision_consistent, desiderata_hold

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
SIGMA_TOL = 1e-4          # |sigma_gpu - sigma_oracle| <= 1e-4 sigma^_1 (FP32 path)


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hd = rk.re_create(0)
    yield hd
    rk.re_destroy(hd)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).cuda()


def oracle_estimate(A, eps, kind, seed, **kw):
    res = alg.rank_estimate(A, eps, kind=kind, seed=seed, **kw)
    res._eps = eps
    return res


# ---------------------------------------------------------------------------
# generator: bit-exact
@pytest.mark.parametrize("n,col0,s", [(1000, 0, 64), (37, 8, 16), (4099, 24, 40)])
def test_gaussian_x_bit_exact(h, n, col0, s):
    out = torch.empty(n, s, dtype=torch.float32, device="cuda")
    rk.re_embedding_x(h, rk.RE_GAUSSIAN, 12345, n, col0, s, out)
    ref = rng.gaussian_x(n, s, 12345, col0).astype(np.float32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("m,row0,r2", [(2048, 0, 128), (333, 16, 48)])
def test_gaussian_y_bit_exact(h, m, row0, r2):
    out = torch.empty(r2, m, dtype=torch.float32, device="cuda")
    rk.re_embedding_y(h, rk.RE_GAUSSIAN, 777, m, row0, r2, out)
    ref = rng.gaussian_y(r2, m, 777, row0).astype(np.float32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("n,col0,s", [(1000, 0, 64), (16384, 8, 32), (5, 0, 8)])
def test_srtt_x_exact(h, n, col0, s):
    out = torch.empty(n, s, dtype=torch.float32, device="cuda")
    rk.re_embedding_x(h, rk.RE_SRHT, 99, n, col0, s, out)
    assert np.array_equal(out.cpu().numpy(), rng.srtt_x(n, s, 99, col0))


@pytest.mark.parametrize("m,row0,r2", [(3000, 0, 64), (64, 8, 48)])
def test_srtt_y_exact(h, m, row0, r2):
    out = torch.empty(r2, m, dtype=torch.float32, device="cuda")
    rk.re_embedding_y(h, rk.RE_SRHT, 5, m, row0, r2, out)
    assert np.array_equal(out.cpu().numpy(), rng.srtt_y(r2, m, 5, row0))


# ---------------------------------------------------------------------------
# right and left sketches: FP32 error bounds against the FP64 oracle
def _right_bound(Ao, X):
    # |fl(A X) - A X| <= gamma_n |A| |X|; FP32 accumulation in K steps of 32 with
    # about n/32 + 32 roundings per entry -> 2 (n/32 + 32) u |A||X| is generous.
    n = Ao.shape[1]
    return 2.0 * (n / 32 + 32) * U32 * (np.abs(Ao) @ np.abs(X)) + 1e-30


@pytest.mark.parametrize("m,n,dtype,kind", [
    (1000, 777, torch.float32, rk.RE_GAUSSIAN),
    (300, 1100, torch.float32, rk.RE_GAUSSIAN),     # m < n: A^T is sketched
    (513, 129, torch.float64, rk.RE_GAUSSIAN),
    (1000, 777, torch.float32, rk.RE_SRHT),
    (257, 3000, torch.float32, rk.RE_SRHT),
    (700, 9000, torch.float32, rk.RE_SRHT),        # transposed
    (9100, 9000, torch.float32, rk.RE_SRHT),       # 2^14-point vectorised transform
    (3001, 2500, torch.float32, rk.RE_SRHT),       # 2^12, ragged row
    (5003, 4100, torch.float32, rk.RE_SRHT),       # 2^13
    (2000, 4097, torch.float32, rk.RE_SRHT),       # row pitch not a multiple of 4: scalar kernel
    (333, 20000, torch.float32, rk.RE_SRHT),       # shared-memory transform (2^15)
])
def test_right_sketch_parity(h, m, n, dtype, kind):
    gen = np.random.default_rng(m * 7 + n)
    A = gen.standard_normal((m, n))
    Ad = dev(A, dtype)
    A_used = Ad.double().cpu().numpy()                   # the values the GPU sees
    Ao, _ = alg.orient(A_used)
    rows, cols = Ao.shape
    for col0, s in ((0, 16), (16, 48)):
        AX = torch.zeros(rows, 64, dtype=torch.float32, device="cuda")
        rk.re_sketch_apply(h, Ad, col0, s, kind, 4242, AX)
        ref = alg.right_sketch(Ao.astype(np.float32).astype(np.float64), s, kind, 4242, col0)
        X = alg.embeddings(kind, cols, rows, s, 4242, col0=col0, r2=0)[0]
        got = AX[:, col0:col0 + s].double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= _right_bound(Ao.astype(np.float32).astype(np.float64), X))
        assert np.all(AX[:, :col0].cpu().numpy() == 0)


def test_srht_row_pitch_padded(h):
    """n not a multiple of 4 inside a wider, aligned row pitch: the register FWHT
    without bulk row copies (the bulk path needs whole 16-byte rows)."""
    m, n, ld = 5000, 4094, 4096                         # m >= n: rows of A are sketched
    gen = np.random.default_rng(17)
    full = gen.standard_normal((m, ld)).astype(np.float32)
    Ad = torch.from_numpy(full).cuda()[:, :n]
    assert Ad.stride(0) == ld
    A64 = full[:, :n].astype(np.float64)
    AX = torch.zeros(m, 32, dtype=torch.float32, device="cuda")
    rk.re_sketch_apply(h, Ad, 0, 32, rk.RE_SRHT, 4242, AX)
    ref = alg.right_sketch(A64, 32, rk.RE_SRHT, 4242, 0)
    X = alg.embeddings(rk.RE_SRHT, n, m, 32, 4242, col0=0, r2=0)[0]
    got = AX.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= _right_bound(A64, X))


@pytest.mark.parametrize("kind", [rk.RE_GAUSSIAN, rk.RE_SRHT])
def test_core_parity_with_appending(h, kind):
    m, n = 2000, 700
    A = np.random.default_rng(3).standard_normal((m, n)).astype(np.float32)
    Ad = dev(A)
    AX = torch.zeros(m, 32, dtype=torch.float32, device="cuda")
    core = torch.zeros(64, 32, dtype=torch.float64, device="cuda")
    rk.re_sketch_apply(h, Ad, 0, 16, kind, 31, AX, core)
    rk.re_sketch_apply(h, Ad, 16, 16, kind, 31, AX, core)
    A64 = A.astype(np.float64)
    ref = alg.core(A64, 32, kind, 31)
    X, Y = alg.embeddings(kind, n, m, 32, 31)
    bound = 4.0 * (m / 32 + n / 32 + 64) * U32 * (np.abs(Y) @ np.abs(A64) @ np.abs(X))
    got = core.cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("m,n,steps", [
    (1_100_000, 12, ((0, 8),)),             # 2^21 padded rows: three transform passes (10 + 10 + 1 bits)
    (3001, 700, ((0, 16), (16, 16), (32, 32))),   # 2^12 rows (10 + 2 bits), appended columns and rows
])
def test_srtt_left_transform_parity(h, m, n, steps):
    """The SRTT left sketch by fast transforms of the columns of D A X, sampled
    at pi_Y(q): the whole core against the oracle's dense S H D (A X) after
    each appending step."""
    A = np.random.default_rng(m).standard_normal((m, n)).astype(np.float32)
    Ad = dev(A)
    c1 = steps[-1][0] + steps[-1][1]
    AX = torch.zeros(m, c1, dtype=torch.float32, device="cuda")
    core = torch.zeros(2 * c1, c1, dtype=torch.float64, device="cuda")
    A64 = A.astype(np.float64)
    for col0, s in steps:
        rk.re_sketch_apply(h, Ad, col0, s, rk.RE_SRHT, 77, AX, core)
        w = col0 + s
        AXg = AX[:, :w].double().cpu().numpy()               # the GPU's right sketch, as the left one saw it
        Y = rng.srtt_y(2 * w, m, 77)
        ref = Y @ AXg
        # FP32 transform: log2(m_pad) levels of additions of +-AX entries
        L = rng.next_pow2_bits(m)
        bound = 2.0 * (L + 2) * U32 * (np.abs(Y) @ np.abs(AXg)) + 1e-30
        got = core[:2 * w, :w].cpu().numpy()
        assert np.all(np.abs(got - ref) <= bound), (col0, s, float(np.max(np.abs(got - ref) / bound)))


@pytest.mark.parametrize("m,n,c0,c1", [
    (3001, 900, 0, 8),          # 16 x 8 core block
    (4099, 1200, 64, 136),      # appended: 144 x 64 and 272 x 72 blocks (two N tiles)
    (2500, 700, 128, 288),      # 320 x 128 and 576 x 160 blocks (three N tiles, two M tiles)
])
def test_core_blocks_parity(h, m, n, c0, c1):
    """Left-sketch blocks of every shape the append step produces, against the
    FP64 oracle's core at the final width."""
    A = np.random.default_rng(m + c1).standard_normal((m, n)).astype(np.float32)
    Ad = dev(A)
    AX = torch.zeros(m, c1, dtype=torch.float32, device="cuda")
    core = torch.zeros(2 * c1, c1, dtype=torch.float64, device="cuda")
    if c0 > 0:
        rk.re_sketch_apply(h, Ad, 0, c0, rk.RE_GAUSSIAN, 57, AX, core)
    rk.re_sketch_apply(h, Ad, c0, c1 - c0, rk.RE_GAUSSIAN, 57, AX, core)
    A64 = A.astype(np.float64)
    ref = alg.core(A64, c1, rk.RE_GAUSSIAN, 57)
    X, Y = alg.embeddings(rk.RE_GAUSSIAN, n, m, c1, 57)
    bound = 4.0 * (m / 32 + n / 32 + 64) * U32 * (np.abs(Y) @ np.abs(A64) @ np.abs(X))
    got = core.cpu().numpy()
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))


@pytest.mark.parametrize("m,n,steps,pad", [
    (3001, 700, ((0, 16), (16, 16), (32, 32)), 0),   # m_pad 4096: appended columns and rows
    (70000, 40, ((0, 8), (8, 24)), 0),               # m_pad 2^17: phases reduced modulo 2^19
    (5000, 300, ((0, 8), (8, 8), (16, 112)), 0),     # 2 c1 = 256 rows: two N tiles of 128
    (3001, 700, ((0, 16), (16, 16)), 1),             # AX rows not 16-byte aligned: CUDA cores
])
def test_srct_left_parity(m, n, steps, pad):
    """The SRCT left embedding (DCT-II rows generated from the cosine table):
    the whole core against the oracle's dense S F D (A X) on the GPU's own A X
    after each appending step.  Aligned A X takes the tensor-core kernel (Y and
    A X as three BF16 terms each), an odd row pitch the CUDA-core kernel."""
    A = np.random.default_rng(m + n).standard_normal((m, n)).astype(np.float32)
    Ad = dev(A)
    c1 = steps[-1][0] + steps[-1][1]
    AX = torch.zeros(m, c1 + pad, dtype=torch.float32, device="cuda")[:, :c1]
    core = torch.zeros(2 * c1, c1, dtype=torch.float64, device="cuda")
    hd = rk.re_create(0, rk.make_opts(y_kind=rk.RE_SRCT))
    try:
        for col0, s in steps:
            rk.re_sketch_apply(hd, Ad, col0, s, rk.RE_GAUSSIAN, 41, AX, core)
            w = col0 + s
            AXg = AX[:, :w].double().cpu().numpy()
            Y = rng.srct_y(2 * w, m, 41)
            ref = Y @ AXg
            # FP32 entries of Y (table values rounded once) and FP32 split-K sums,
            # bounded as the Gaussian core blocks are
            bound = 4.0 * (m / 32 + 64) * U32 * (np.abs(Y) @ np.abs(AXg)) + 1e-30
            got = core[:2 * w, :w].cpu().numpy()
            assert np.all(np.abs(got - ref) <= bound), (col0, s, float(np.max(np.abs(got - ref) / bound)))
    finally:
        rk.re_destroy(hd)


@pytest.mark.parametrize("precision", [rk.RE_PREC_FP32, rk.RE_PREC_BF16X3])
def test_srct_left_rank_estimate(precision):
    """Gaussian X with the SRCT Y (the paper's experimental pairing for the rank
    estimate, Sec. 6.1): the oracle's rank, width and sketched values on a gap."""
    sig = wl.spectrum("step", 700, rank=45, tail_scale=1e-9)
    A = wl.haar_matrix(2500, 700, sig, seed=13).numpy().astype(np.float32)
    hd = rk.re_create(0, rk.make_opts(precision=precision, y_kind=rk.RE_SRCT))
    try:
        res, sg = rk.re_rank_estimate(hd, dev(A), 1e-5, rk.RE_GAUSSIAN, 19, sigma_cap=512)
    finally:
        rk.re_destroy(hd)
    orc = alg.rank_estimate(A.astype(np.float64), 1e-5, kind=alg.GAUSSIAN, seed=19, ykind=alg.SRCT)
    assert orc.converged and (res.rank, res.final_s) == (orc.rank, orc.final_s) == (45, 64)
    assert np.max(np.abs(sg[:res.n_sigma] - orc.sigma)) <= 1e-4 * orc.sigma[0]


def test_srct_y_kind_errors():
    with pytest.raises(rk.RankEstError) as e:
        rk.re_create(0, rk.make_opts(y_kind=rk.RE_HRTT))
    assert e.value.code == rk.RE_ERR_ARG


def test_core_sigma_against_lapack(h):
    for (r2, s, seed) in ((16, 8, 0), (128, 64, 1), (256, 128, 2), (512, 256, 3), (37, 29, 4),
                          (1024, 512, 5), (600, 300, 6), (1000, 70, 7)):
        gen = np.random.default_rng(seed)
        U, _ = np.linalg.qr(gen.standard_normal((r2, s)))
        V, _ = np.linalg.qr(gen.standard_normal((s, s)))
        sv = np.logspace(0, -9, s)
        C = (U * sv) @ V.T
        sig = torch.zeros(s, dtype=torch.float64, device="cuda")
        rk.re_core_sigma(h, dev(C, torch.float64), sig)
        got = sig.cpu().numpy()
        ref = np.linalg.svd(C, compute_uv=False)
        assert np.all(np.diff(got) <= 0)
        # FP32 one-sided Jacobi: each column takes ~sweeps*(s-1) rotations, each
        # rounding its entries once (~u relative), so |error| ~ 2u sqrt(8 s) sigma_1;
        # 3e-5 sigma_1 covers s <= 512 (input rounding to FP32 adds ~u sigma_1).
        assert np.max(np.abs(got - ref)) <= 3e-5 * ref[0], (r2, s, np.max(np.abs(got - ref)))


# ---------------------------------------------------------------------------
# end-to-end Algorithm 1
def check_estimate(h, A_host, eps, kind, seed, dtype=torch.float32, exact=True, **kw):
    Ad = dev(A_host, dtype)
    A_used = Ad.double().cpu().numpy()
    if dtype == torch.float64:
        A_used = A_used.astype(np.float32).astype(np.float64)   # FP64 input is read as FP32
    res, sig = rk.re_rank_estimate(h, Ad, eps, kind, seed)
    orc = oracle_estimate(A_used, eps, kind, seed, **kw)
    assert res.final_s == orc.final_s or not exact
    n = min(len(sig), len(orc.sigma))
    assert np.max(np.abs(sig[:n] - orc.sigma[:n])) <= SIGMA_TOL * orc.sigma[0]
    if exact:
        assert res.rank == orc.rank
    else:
        assert decision_consistent(res.rank, res.final_s, sig, A_used, eps, kind, seed,
                                   converged=bool(res.flags & rk.RE_CONVERGED), **kw), (res.rank, orc.rank)
    assert bool(res.flags & rk.RE_CONVERGED) == orc.converged
    assert bool(res.flags & rk.RE_TRANSPOSED) == orc.transposed
    return res, orc


def test_small_fp64_decade_spectrum(h):
    # 2048 x 1024 FP64, sigma_i = 10^{-(i-1)/10} (i <= 60) then 1e-12, eps = 1e-4:
    # sigma_41 sits exactly on the threshold, so +-1 is legitimate near it.
    sig = wl.spectrum("decade10", 1024)
    A = wl.haar_matrix(2048, 1024, sig, seed=0).numpy()
    res, orc = check_estimate(h, A, 1e-4, rk.RE_GAUSSIAN, 12345, dtype=torch.float64, exact=False)
    assert res.final_s == 64 and res.passes == 4
    # no clear gap near eps: the Sec. 1.1 desiderata bound the answer
    s = sig.numpy()
    assert s[res.rank] < 10 * 1e-4 and s[res.rank - 1] > 0.1 * 1e-4


@pytest.mark.parametrize("kind", [rk.RE_GAUSSIAN, rk.RE_SRHT, rk.RE_HRTT])
@pytest.mark.parametrize("m,n,rank", [(1500, 600, 37), (600, 1500, 37), (4096, 4096, 120),
                                      (333, 257, 5), (2000, 1000, 0)])
def test_clear_gap_exact_rank(h, kind, m, n, rank):
    k = min(m, n)
    sig = wl.spectrum("step", k, rank=rank, tail_scale=1e-9) if rank else torch.full((k,), 1e-30)
    A = wl.haar_matrix(m, n, sig, seed=rank + m).numpy()
    if rank == 0:
        A = np.zeros((m, n))
    res, orc = check_estimate(h, A, 1e-4, kind, 7 + rank)
    assert res.rank == rank


@pytest.mark.parametrize("fam,eps", [("fe", 1e-6), ("fp", 1e-4), ("sp", 1e-2)])
def test_ungapped_families(h, fam, eps):
    sig = wl.spectrum(fam, 800)
    A = wl.haar_matrix(1200, 800, sig, seed=11).numpy()
    res, orc = check_estimate(h, A, eps, rk.RE_GAUSSIAN, 3, exact=False)
    s = sig.numpy()
    r = res.rank
    assert s[r] < 10 * eps * s[0] and (r == 0 or s[r - 1] > 0.1 * eps * s[0])


def test_tiny_and_ragged(h):
    for (m, n, rank) in ((33, 17, 3), (17, 33, 3), (100, 1, 1), (257, 129, 20)):
        sig = wl.spectrum("step", min(m, n), rank=rank, tail_scale=1e-10)
        A = wl.haar_matrix(m, n, sig, seed=m).numpy()
        res, orc = check_estimate(h, A, 1e-5, rk.RE_GAUSSIAN, 1)
        assert res.rank == rank


def test_lower_bound_when_capped(h):
    sig = wl.spectrum("step", 500, rank=100, tail_scale=1e-9)
    A = wl.haar_matrix(900, 500, sig, seed=1).numpy()
    o = rk.make_opts(s_max=64)
    rk.re_set_opts(h, o)
    try:
        res, sig_g = rk.re_rank_estimate(h, dev(A), 1e-4, rk.RE_GAUSSIAN, 2)
    finally:
        rk.re_set_opts(h, rk.re_opts_default())
    assert res.flags & rk.RE_LOWER_BOUND_ONLY and res.rank == 58 and res.final_s == 64


def test_host_entry_point_matches_device(h):
    sig = wl.spectrum("step", 512, rank=30, tail_scale=1e-9)
    A = wl.haar_matrix(1024, 512, sig, seed=4).numpy().astype(np.float32)
    r1, s1 = rk.re_rank_estimate(h, dev(A), 1e-4, rk.RE_GAUSSIAN, 9)
    r2, s2 = rk.re_rank_estimate_host(h, A, 1e-4, rk.RE_GAUSSIAN, 9)
    assert r1.rank == r2.rank == 30 and np.array_equal(s1, s2)


@pytest.mark.parametrize("precision", [rk.RE_PREC_BF16X3, rk.RE_PREC_FP32])
def test_first_width_and_pipelined_host_path(precision):
    """A wide first pass (opts.first_width) and the host entry point's chunked
    copy with the first pass under it return the plain ladder's rank and width,
    sigma within the small-core SVD's accuracy, in fewer passes over A."""
    sig = wl.spectrum("step", 2048, rank=150, tail_scale=1e-9)
    A = wl.haar_matrix(8192, 2048, sig, seed=6).to(torch.float32)
    Ad = A.cuda()
    hp = rk.re_create(0, rk.make_opts(precision=precision))
    hw = rk.re_create(0, rk.make_opts(precision=precision, first_width=128))
    try:
        r0, s0 = rk.re_rank_estimate(hp, Ad, 1e-4, rk.RE_GAUSSIAN, 3, sigma_cap=512)
        r1, s1 = rk.re_rank_estimate(hw, Ad, 1e-4, rk.RE_GAUSSIAN, 3, sigma_cap=512)
        hh = rk.re_create(0, rk.make_opts(precision=precision, first_width=256))
        r2, s2 = rk.re_rank_estimate_host(hh, A.numpy(), 1e-4, rk.RE_GAUSSIAN, 3, sigma_cap=512)
        r3, s3 = rk.re_rank_estimate_host(hh, A.numpy(), 1e-4, rk.RE_GAUSSIAN, 3, sigma_cap=512)
        rk.re_destroy(hh)
        r4, s4 = rk.re_rank_estimate_host(hp, A.numpy(), 1e-4, rk.RE_GAUSSIAN, 3, sigma_cap=512)
    finally:
        rk.re_destroy(hp)
        rk.re_destroy(hw)
    assert r0.rank == 150 and r0.final_s == 256 and r0.passes == 6
    for r, sg in ((r1, s1), (r2, s2), (r3, s3), (r4, s4)):
        assert (r.rank, r.final_s, r.flags, r.n_sigma) == (r0.rank, r0.final_s, r0.flags, r0.n_sigma)
        # A X differs by FP32 rounding; the FP32 small-core SVD holds sigma to about
        # 1e-5 sigma_1 (its stop rule), the bound used for it against LAPACK
        assert np.max(np.abs(sg[:r0.n_sigma] - s0[:r0.n_sigma])) <= 3e-5 * s0[0]
    assert r1.passes == 2          # 128 columns, then 128 more
    assert r2.passes == 1 and r3.passes == 1   # 256 columns sketched under the copy
    assert r4.passes == r0.passes              # plain ladder, its first pass under the copy
    assert np.array_equal(s2, s3)  # the chunked path is deterministic


def test_handles_on_concurrent_host_threads():
    """Handles are independent: host threads, each with its own handle and
    stream, estimating matrices of different shapes at the same time (so the
    kernels' dynamic shared memory differs between concurrent launches) get
    exactly the results of one thread running them in turn."""
    import concurrent.futures as cf
    shapes = [(4096, 1024, 60), (2048, 512, 30), (3000, 700, 45), (1024, 1024, 80)]
    mats = []
    for i, (m, n, r) in enumerate(shapes):
        sig = wl.spectrum("step", n, rank=r, tail_scale=1e-9)
        mats.append(wl.haar_matrix(m, n, sig, seed=20 + i).to(torch.float32).cuda())
    opts = rk.make_opts(precision=rk.RE_PREC_BF16X3)

    def run(j, reps):
        hd = rk.re_create(0, opts)
        st = torch.cuda.Stream()
        out = []
        try:
            for _ in range(reps):
                res, sg = rk.re_rank_estimate(hd, mats[j], 1e-5, rk.RE_GAUSSIAN, 7 + j, sigma_cap=256, stream=st)
                out.append((res.rank, res.final_s, res.flags, sg.copy()))
        finally:
            rk.re_destroy(hd)
        return out

    ref = [run(j, 1)[0] for j in range(len(mats))]
    with cf.ThreadPoolExecutor(max_workers=len(mats)) as ex:
        got = list(ex.map(lambda j: run(j, 6), range(len(mats))))
    for j, (m, n, r) in enumerate(shapes):
        assert ref[j][0] == r
        for res in got[j]:
            assert res[:3] == ref[j][:3] and np.array_equal(res[3], ref[j][3])


def test_first_width_option_errors():
    with pytest.raises(rk.RankEstError) as e:
        rk.re_create(0, rk.make_opts(first_width=12))
    assert e.value.code == rk.RE_ERR_ARG
    with pytest.raises(rk.RankEstError) as e:
        rk.re_create(0, rk.make_opts(first_width=64, learned=1))
    assert e.value.code == rk.RE_ERR_ARG


def test_errors(h):
    A = torch.ones(64, 32, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate(h, A, 0.0)
    assert e.value.code == rk.RE_ERR_ARG
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate(h, A, 1e-3, m=64, n=32, ld=16, dtype=rk.RE_F32)
    assert e.value.code == rk.RE_ERR_ARG
    B = torch.randn(300, 200, device="cuda")
    B[17, 3] = float("nan")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate(h, B, 1e-3)
    assert e.value.code == rk.RE_ERR_NONFINITE
    B[17, 3] = float("inf")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate(h, B, 1e-3)
    assert e.value.code == rk.RE_ERR_NONFINITE
    # the handle still works after an error
    res, _ = rk.re_rank_estimate(h, torch.zeros(64, 32, device="cuda"), 1e-3)
    assert res.rank == 0


def test_batched_kernel_blocks(h):
    shapes = wl.kernel_block_sizes(6, seed=3, lo=256, hi=1024)
    blocks = [wl.kernel_block(m, n, seed=100 + i).cuda() for i, (m, n) in enumerate(shapes)]
    res, sig = rk.re_rank_estimate_batched(h, blocks, 1e-6, rk.RE_GAUSSIAN, 500, sigma_cap=512)
    for i, B in enumerate(blocks):
        Ah = B.double().cpu().numpy()
        orc = oracle_estimate(Ah, 1e-6, alg.GAUSSIAN, 500 + i)
        assert res[i].status == 0
        if res[i].final_s == orc.final_s:
            n = min(res[i].n_sigma, len(orc.sigma))
            assert np.max(np.abs(sig[i, :n] - orc.sigma[:n])) <= SIGMA_TOL * orc.sigma[0]
        k = res[i].n_sigma
        assert decision_consistent(res[i].rank, res[i].final_s, sig[i, :k], Ah, 1e-6, alg.GAUSSIAN, 500 + i,
                                   converged=bool(res[i].flags & rk.RE_CONVERGED)), (i, res[i].rank, orc.rank)
        assert desiderata_hold(res[i].rank, Ah, 1e-6)


# ---------------------------------------------------------------------------
# HRTT (Sec. 3.4): hashed randomized Hadamard right sketch
@pytest.mark.parametrize("n,s", [(1000, 64), (37, 24), (4099, 40), (256, 256)])
def test_hrtt_x_exact(h, n, s):
    out = torch.empty(n, s, dtype=torch.float32, device="cuda")
    rk.re_embedding_x(h, rk.RE_HRTT, 77, n, 0, s, out)
    assert np.array_equal(out.cpu().numpy(), rng.hrtt_x(n, s, 77))


def _hrtt_bounds(Ao, s):
    """Per-entry bounds for the FP32 HRTT sketch of the rows a of Ao.

    Rigorous: each transformed value is a sum of +-a_i over L = log2 n_pad
    levels and a bucket adds b <= ceil(n_pad / s) of them, so in any order of
    additions |err| <= (L + b) b u ||a||_1 (doubled).  Discriminating: an
    output is typically sqrt(b) ||a||_2 in size and one wrong or missing term
    moves it by about ||a||_2, while rounding moves it by about
    u sqrt(L + b) sqrt(b) ||a||_2; 1e-3 sqrt(b) ||a||_2 separates the two."""
    L = rng.next_pow2_bits(Ao.shape[1])
    b = -(-(1 << L) // s)
    l1 = np.abs(Ao).sum(axis=1)[:, None]
    l2 = np.sqrt((Ao * Ao).sum(axis=1))[:, None]
    return 2.0 * (L + b) * b * U32 * l1 + 1e-30, 1e-3 * np.sqrt(b) * l2 + 1e-30


@pytest.mark.parametrize("m,n,dtype,widths", [
    (1000, 777, torch.float32, (16, 24, 64)),       # 2^10 register transform, sums per output
    (300, 1100, torch.float32, (16,)),              # m < n: A^T is sketched
    (513, 129, torch.float64, (8, 24)),             # FP64 input (read as FP32)
    (3001, 2500, torch.float32, (16, 64, 256)),     # 2^12 bulk rows: s < 32, 32 <= s < T, s > T
    (5003, 4100, torch.float32, (24, 128)),         # 2^13: width not a power of two, then bulk
    (9100, 9000, torch.float32, (16, 512)),         # 2^14 bulk rows, s = T
    (2000, 4097, torch.float32, (16,)),             # row pitch not a multiple of 4
])
def test_hrtt_right_sketch_parity(h, m, n, dtype, widths):
    gen = np.random.default_rng(m * 11 + n)
    A = gen.standard_normal((m, n))
    Ad = dev(A, dtype)
    Ao, _ = alg.orient(Ad.double().cpu().numpy())
    Ao = Ao.astype(np.float32).astype(np.float64)        # the values the kernels add
    rows = Ao.shape[0]
    for s in widths:
        AX = torch.zeros(rows, s, dtype=torch.float32, device="cuda")
        rk.re_sketch_apply(h, Ad, 0, s, rk.RE_HRTT, 4242, AX)
        ref = alg.right_sketch(Ao, s, rk.RE_HRTT, 4242)
        err = np.abs(AX.double().cpu().numpy() - ref)
        rigorous, tight = _hrtt_bounds(Ao, s)
        assert np.all(err <= rigorous) and np.all(err <= tight), (s, float(np.max(err / tight)))


def test_hrtt_shared_memory_transform(h):
    """2^15-point rows (16400 columns, one row per CTA): A is zero outside 48
    columns (the last one among them), so the oracle needs only those rows of X."""
    m = n = 16400
    gen = np.random.default_rng(5)
    nz = np.sort(np.append(gen.choice(n - 1, 47, replace=False), n - 1))
    vals = gen.standard_normal((m, nz.size)).astype(np.float32)
    Ad = torch.zeros(m, n, dtype=torch.float32, device="cuda")
    Ad[:, torch.from_numpy(nz).cuda()] = torch.from_numpy(vals).cuda()
    Asub = vals.astype(np.float64)
    for s in (16, 40):
        AX = torch.zeros(m, s, dtype=torch.float32, device="cuda")
        rk.re_sketch_apply(h, Ad, 0, s, rk.RE_HRTT, 99, AX)
        ref = Asub @ rng.hrtt_x(n, s, 99, rows=nz)
        err = np.abs(AX.double().cpu().numpy() - ref)
        b = -(-(1 << 15) // s)
        l1 = np.abs(Asub).sum(axis=1)[:, None]
        l2 = np.sqrt((Asub * Asub).sum(axis=1))[:, None]
        assert np.all(err <= 2.0 * (15 + b) * b * U32 * l1) and np.all(err <= 1e-3 * np.sqrt(b) * l2)
    del Ad
    torch.cuda.empty_cache()


def test_hrtt_core_parity(h):
    # the whole width-s sketch and its 2s x s core (Gaussian Y) in one call
    m, n, s = 2000, 700, 32
    A = np.random.default_rng(8).standard_normal((m, n)).astype(np.float32)
    AX = torch.zeros(m, s, dtype=torch.float32, device="cuda")
    core = torch.zeros(2 * s, s, dtype=torch.float64, device="cuda")
    rk.re_sketch_apply(h, dev(A), 0, s, rk.RE_HRTT, 31, AX, core)
    A64 = A.astype(np.float64)
    ref = alg.core(A64, s, rk.RE_HRTT, 31)
    Y = alg.embeddings(rk.RE_HRTT, n, m, s, 31)[1]
    b = -(-1024 // s)
    # |AX entries| error as above, then FP32 accumulation of the left sketch
    ax_abs = (np.abs(A64).sum(axis=1) * b)[:, None] * np.ones((1, s))
    bound = 4.0 * (m / 32 + 10 + b + 64) * U32 * (np.abs(Y) @ ax_abs)
    assert np.all(np.abs(core.cpu().numpy() - ref) <= bound)


def test_hrtt_coherent_diagonal(h):
    """Sec. 3.4: on a diagonal matrix the hashed transform keeps the exact rank
    (and the oracle's sigma), while the sampled one falls short."""
    n = 2048
    A = np.diag(np.where(np.arange(n) < 150, 1.0, 1e-8))
    res, orc = check_estimate(h, A, 1e-4, rk.RE_HRTT, 5)
    assert res.rank == 150 and res.final_s == 256 and res.passes == 6 and res.gap_index == 150
    res_s, _ = rk.re_rank_estimate(h, dev(A), 1e-4, rk.RE_SRHT, 5)
    assert res_s.rank < 150


def test_hrtt_errors(h):
    A = torch.randn(300, 100, device="cuda")
    AX = torch.zeros(300, 64, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply(h, A, 8, 8, rk.RE_HRTT, 1, AX)          # not appendable
    assert e.value.code == rk.RE_ERR_ARG
    AX = torch.zeros(300, 256, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply(h, A, 0, 256, rk.RE_HRTT, 1, AX)        # s > n_pad = 128
    assert e.value.code == rk.RE_ERR_ARG
    # full column rank 100: at s = 128 (r1 = 116) the core has rank 100 and the
    # read-off finds sigma_101 at the rounding level
    res, _ = rk.re_rank_estimate(h, A, 1e-3, rk.RE_HRTT, 1)
    assert res.rank == 100 and res.flags & rk.RE_CONVERGED and res.final_s == 128


# ---------------------------------------------------------------------------
# step 7 by the QR diagonal (the remark after Algorithm 1, Sec. 5)
@pytest.mark.parametrize("m,n,rank", [(1500, 600, 37), (3000, 1200, 200), (600, 1500, 60)])
def test_qr_diagonal_estimate(h, m, n, rank):
    """|R_kk| of the core's QR as the singular-value estimates: the GPU's FP32
    Householder QR against the oracle's LAPACK QR of the FP64 core (within 1e-4
    sigma^_1, the FP32 tolerance), and the oracle's rank on a clear gap; rank 200
    ends at s = 256, where the core is factored by the cluster QR kernel."""
    sig = wl.spectrum("step", min(m, n), rank=rank, tail_scale=1e-9)
    A = wl.haar_matrix(m, n, sig, seed=rank + 5).numpy()
    Ad = dev(A)
    rk.re_set_opts(h, rk.make_opts(sigma_est=rk.RE_SIGMA_QRDIAG))
    try:
        res, sg = rk.re_rank_estimate(h, Ad, 1e-4, rk.RE_GAUSSIAN, 3)
    finally:
        rk.re_set_opts(h, rk.re_opts_default())
    orc = alg.rank_estimate(Ad.double().cpu().numpy(), 1e-4, kind=alg.GAUSSIAN, seed=3, sigma="qrdiag")
    assert res.rank == orc.rank == rank and res.final_s == orc.final_s
    k = min(len(sg), len(orc.sigma))
    assert np.max(np.abs(sg[:k] - orc.sigma[:k])) <= SIGMA_TOL * orc.sigma[0]
    assert res.svd_sweeps == 0
