"""Parity of the BF16x3 tensor-core (tcgen05) right sketch with the FP64 oracle.

A is split exactly into three BF16 terms and X entries are BF16-exact, so every
product is exact and only FP32 accumulation (in TMEM) rounds: the same
|A||X|-scaled bound as the FP32 path applies.
"""
import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def htc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    h = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    yield h
    rk.re_destroy(h)


@pytest.mark.parametrize("m,n,col0,s", [
    (128, 64, 0, 16),        # one tile, one K chunk
    (300, 100, 0, 8),        # ragged M and K, N padded 8 -> 16
    (1000, 777, 16, 48),     # several tiles, ragged K chunk
    (2049, 1030, 0, 128),
    (513, 300, 8, 256),      # N = 256, two pipeline stages
    (5000, 4096, 64, 64),
    (19584, 1024, 0, 32),    # 153 row tiles on 152 SMs: tiles shared by two CTAs
    (20400, 1000, 8, 128),   # 160 tiles, ragged last tile and K chunk, shared tiles
])
def test_tc_right_sketch_parity(htc, m, n, col0, s):
    A = np.random.default_rng(m + n + s).standard_normal((m, n)).astype(np.float32)
    A[0, :5] = [1e-30, -3e-20, 1e20, 7.0, -0.0]          # wide exponent range stays exact
    Ad = torch.from_numpy(A).cuda()
    AX = torch.zeros(m, col0 + s, dtype=torch.float32, device="cuda")
    rk.re_sketch_apply(htc, Ad, col0, s, rk.RE_GAUSSIAN, 99, AX)
    A64 = A.astype(np.float64)
    ref = alg.right_sketch(A64, s, alg.GAUSSIAN, 99, col0)
    X = alg.embeddings(alg.GAUSSIAN, n, m, s, 99, col0=col0, r2=0)[0]
    bound = 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
    got = AX[:, col0:].double().cpu().numpy()
    err = np.abs(got - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.all(AX[:, :col0].cpu().numpy() == 0)


def test_tc_matches_fp32_path_closely(htc):
    m, n = 4096, 2048
    A = np.random.default_rng(5).standard_normal((m, n)).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    h32 = rk.re_create(0)
    try:
        a1 = torch.zeros(m, 64, device="cuda")
        a2 = torch.zeros(m, 64, device="cuda")
        rk.re_sketch_apply(htc, Ad, 0, 64, rk.RE_GAUSSIAN, 3, a1)
        rk.re_sketch_apply(h32, Ad, 0, 64, rk.RE_GAUSSIAN, 3, a2)
    finally:
        rk.re_destroy(h32)
    rel = (a1 - a2).abs().max() / a2.abs().max()
    assert rel < 1e-5


@pytest.mark.parametrize("m,n,rank", [(1500, 600, 37), (4096, 4096, 120), (600, 1500, 37)])
def test_tc_rank_estimate_clear_gap(htc, m, n, rank):
    sig = wl.spectrum("step", min(m, n), rank=rank, tail_scale=1e-9)
    A = wl.haar_matrix(m, n, sig, seed=rank + m).to(torch.float32)
    res, sg = rk.re_rank_estimate(htc, A.cuda(), 1e-4, rk.RE_GAUSSIAN, 7 + rank)
    orc = alg.rank_estimate(A.double().numpy(), 1e-4, kind=alg.GAUSSIAN, seed=7 + rank)
    assert res.rank == orc.rank == rank and res.final_s == orc.final_s
    k = min(len(sg), len(orc.sigma))
    assert np.max(np.abs(sg[:k] - orc.sigma[:k])) <= 1e-4 * orc.sigma[0]


def test_tc_shared_tiles_deterministic(htc):
    """Tiles split between two CTAs are summed by two additions onto zero: the
    result is the same bit pattern on every call."""
    m, n, s = 39000, 1100, 64                 # 305 row tiles: most CTAs share a tile
    A = torch.from_numpy(np.random.default_rng(11).standard_normal((m, n)).astype(np.float32)).cuda()
    outs = []
    for _ in range(3):
        AX = torch.full((m, s), float("nan"), dtype=torch.float32, device="cuda")
        rk.re_sketch_apply(htc, A, 0, s, rk.RE_GAUSSIAN, 21, AX)
        outs.append(AX)
    assert torch.isfinite(outs[0]).all()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])


def test_tc_bounded_wait_expires_and_context_survives():
    """Failure path: with the test hook one CTA withholds its first A tile, so the
    waits on it expire (bounded, about 2 s); every role drains and frees TMEM, the
    estimate reports RE_ERR_TIMEOUT, and the next estimate on the same handle (same
    CUDA context) is correct."""
    import time
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    rank = 20
    sig = wl.spectrum("step", 2048, rank=rank, tail_scale=1e-9)
    A = wl.haar_matrix(4096, 2048, sig, seed=3).to(torch.float32).cuda()
    h = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3, test_drop_load=1))
    try:
        t0 = time.time()
        with pytest.raises(rk.RankEstError) as e:
            rk.re_rank_estimate(h, A, 1e-4, rk.RE_GAUSSIAN, 3)
        assert e.value.code == rk.RE_ERR_TIMEOUT
        assert time.time() - t0 < 60
        rk.re_set_opts(h, rk.make_opts(precision=rk.RE_PREC_BF16X3))
        res, _ = rk.re_rank_estimate(h, A, 1e-4, rk.RE_GAUSSIAN, 3)
        assert res.status == 0 and res.rank == rank
    finally:
        rk.re_destroy(h)
    torch.cuda.synchronize()


@pytest.mark.parametrize("m,n,col0,s", [
    (300, 100, 0, 8),        # ragged M and K, n_pad 128
    (1000, 777, 16, 48),     # appended columns
    (2049, 1030, 0, 128),
    (513, 300, 8, 256),      # N = 256
    (20400, 1000, 8, 128),   # shared tiles
])
def test_tc_srht_right_sketch_parity(htc, m, n, col0, s):
    """With BF16x3 precision the SRHT's sampled columns (X = D H S^T, +-1 entries,
    exact in BF16) go through the tensor-core contraction: the oracle's dense
    S H D product within the FP32 accumulation bound."""
    A = np.random.default_rng(m + n + s + 1).standard_normal((m, n)).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    AX = torch.zeros(m, col0 + s, dtype=torch.float32, device="cuda")
    rk.re_sketch_apply(htc, Ad, col0, s, rk.RE_SRHT, 99, AX)
    A64 = A.astype(np.float64)
    ref = alg.right_sketch(A64, s, alg.SRHT, 99, col0)
    X = alg.embeddings(alg.SRHT, n, m, s, 99, col0=col0, r2=0)[0]
    bound = 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
    err = np.abs(AX[:, col0:].double().cpu().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_tc_srht_rank_matches_transform_path(htc):
    """The tensor-core SRHT and the register-transform SRHT compute the same sketch
    up to FP32 rounding: same rank, width and passes on a clear gap, sigma within
    the small-core SVD's accuracy; both equal to the oracle's rank."""
    sig = wl.spectrum("step", 1500, rank=70, tail_scale=1e-9)
    A = wl.haar_matrix(4000, 1500, sig, seed=31).to(torch.float32)
    Ad = A.cuda()
    r_tc, s_tc = rk.re_rank_estimate(htc, Ad, 1e-5, rk.RE_SRHT, 8)
    h32 = rk.re_create(0)
    try:
        r_fw, s_fw = rk.re_rank_estimate(h32, Ad, 1e-5, rk.RE_SRHT, 8)
    finally:
        rk.re_destroy(h32)
    orc = alg.rank_estimate(A.double().numpy(), 1e-5, kind=alg.SRHT, seed=8)
    assert (r_tc.rank, r_tc.final_s, r_tc.passes) == (r_fw.rank, r_fw.final_s, r_fw.passes) == \
        (orc.rank, orc.final_s, orc.passes)
    assert np.max(np.abs(s_tc[:r_tc.n_sigma] - s_fw[:r_fw.n_sigma])) <= 3e-5 * s_fw[0]


@pytest.mark.parametrize("m,n,s", [
    (300, 1000, 8),          # m < n: transposed, the register transform (not the tensor-core path)
    (2000, 1000, 8),         # n_pad 1024 <= 256 s: one BF16 plane of X
    (3001, 3000, 16),        # 4096, buckets of 256
    (9100, 9000, 64),        # 16384, buckets of 256
    (5000, 5000, 512),       # 8192: two launches of 256 columns
    (9000, 4000, 8),         # 4096 > 256 s: buckets of 512, two planes (BF16 and remainder)
    (9100, 9000, 32),        # 16384: buckets of 512, two planes
    (5000, 20000, 16),       # transposed, 2^15: the register transform
])
def test_tc_hrtt_right_sketch_parity(htc, m, n, s):
    """With BF16x3 precision the HRTT's dense X = D H C^T (integer entries of
    magnitude at most the bucket size) goes through the tensor-core contraction:
    one exact BF16 plane for buckets of at most 256 coordinates, a BF16 and its
    exact remainder otherwise.  The oracle's X within the FP32 accumulation bound."""
    A = np.random.default_rng(m + n + s + 2).standard_normal((m, n)).astype(np.float32)
    Ad = torch.from_numpy(A).cuda()
    A64 = A.astype(np.float64)
    Ao, _ = alg.orient(A64)
    rows, cols = Ao.shape
    AX = torch.zeros(rows, s, dtype=torch.float32, device="cuda")
    rk.re_sketch_apply(htc, Ad, 0, s, rk.RE_HRTT, 61, AX)
    ref = alg.right_sketch(Ao, s, alg.HRTT, 61)
    X = alg.embeddings(alg.HRTT, cols, rows, s, 61, r2=0)[0]
    bound = 2.0 * (cols / 16 + 32) * U32 * (np.abs(Ao) @ np.abs(X)) + 1e-35
    err = np.abs(AX.double().cpu().numpy() - ref)
    assert np.all(err <= bound), float(np.max(err / bound))
