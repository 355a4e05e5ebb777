"""Batched Algorithm 1 (one captured graph over many uneven blocks) against the
FP64 oracle run block by block, and against the single-matrix entry point."""
import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

from rankcheck import decision_consistent, desiderata_hold

pytestmark = pytest.mark.gpu
SIGMA_TOL = 1e-4
PREC = {}          # handle -> precision of the fixture that made it


def expected_passes(h, final_s, s0=8):
    """Passes over a block that stopped at width final_s: one per ladder width on
    the CUDA cores; on the tensor cores the first pass appends up to 4 s0 columns
    (here 32, within the X^T pool of s_max / 2 = 64 rows), then one per width."""
    w1 = s0 if PREC[h] != rk.RE_PREC_BF16X3 else 4 * s0
    passes, t = 1, 2 * w1
    while t <= final_s:
        passes += 1
        t *= 2
    return passes


@pytest.fixture(scope="module", params=[rk.RE_PREC_FP32, rk.RE_PREC_BF16X3], ids=["fp32", "bf16x3"])
def h(request):
    """FP32 CUDA-core sketch and BF16x3 tensor-core sketch (4-byte asynchronous
    copies, any row pitch, transposed blocks included)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    # the tensor-core ladder's first pass pinned to 32 columns (autotuned by default,
    # tested separately below), so that the pass counts are known
    hd = rk.re_create(0, rk.make_opts(s_max=128, precision=request.param,
                                      batch_first_width=32 if request.param == rk.RE_PREC_BF16X3 else 0))
    PREC[hd] = request.param
    yield hd
    rk.re_destroy(hd)


def _decision_ok(r, sig_row, A, eps, seed, s_max=128):
    """The block's rank and final width follow from the oracle's sketched values up
    to decisions inside the error measured on this block (tests/rankcheck.py), and
    the Sec. 1.1 desiderata hold against the block's exact singular values."""
    k = r.n_sigma
    return (decision_consistent(r.rank, r.final_s, sig_row[:k], A, eps, alg.GAUSSIAN, seed, s_max=s_max,
                                converged=bool(r.flags & rk.RE_CONVERGED))
            and desiderata_hold(r.rank, A, eps))


def test_batched_gapped_blocks_exact(h):
    # clear gaps, uneven and transposed shapes: ranks identical to the oracle's
    specs = [(300, 257, 5), (257, 700, 12), (1024, 1024, 40), (900, 300, 1), (333, 333, 70),
             (2000, 600, 100), (600, 2000, 3), (512, 256, 0)]
    blocks, mats = [], []
    for i, (m, n, r) in enumerate(specs):
        k = min(m, n)
        if r == 0:
            A = torch.zeros(m, n, dtype=torch.float64)
        else:
            A = wl.haar_matrix(m, n, wl.spectrum("step", k, rank=r, tail_scale=1e-9), seed=i)
        A32 = A.to(torch.float32)
        blocks.append(A32.cuda())
        mats.append(A32.double().numpy())
    res, sig = rk.re_rank_estimate_batched(h, blocks, 1e-4, rk.RE_GAUSSIAN, 900, sigma_cap=128)
    for i, (m, n, r) in enumerate(specs):
        orc = alg.rank_estimate(mats[i], 1e-4, kind=alg.GAUSSIAN, seed=900 + i, s_max=128)
        assert res[i].status == 0
        assert res[i].rank == orc.rank == r, (i, res[i].rank, orc.rank)
        assert res[i].final_s == orc.final_s
        assert res[i].passes == expected_passes(h, res[i].final_s)
        assert orc.passes == expected_passes(h, orc.final_s) or PREC[h] == rk.RE_PREC_BF16X3
        k = min(res[i].n_sigma, len(orc.sigma))
        assert np.max(np.abs(sig[i, :k] - orc.sigma[:k])) <= SIGMA_TOL * max(orc.sigma[0], 1e-300)
        assert bool(res[i].flags & rk.RE_TRANSPOSED) == (m < n)


def test_batched_kernel_blocks_and_replay(h):
    shapes = wl.kernel_block_sizes(24, seed=11, lo=256, hi=2048)
    blocks = [wl.kernel_block(m, n, seed=300 + i).cuda() for i, (m, n) in enumerate(shapes)]
    r1, s1 = rk.re_rank_estimate_batched(h, blocks, 1e-6, rk.RE_GAUSSIAN, 77, sigma_cap=128)
    r2, s2 = rk.re_rank_estimate_batched(h, blocks, 1e-6, rk.RE_GAUSSIAN, 77, sigma_cap=128)   # graph replay
    assert [x.rank for x in r1] == [x.rank for x in r2] and np.array_equal(s1, s2)
    for i, B in enumerate(blocks):
        Ah = B.double().cpu().numpy()
        orc = alg.rank_estimate(Ah, 1e-6, kind=alg.GAUSSIAN, seed=77 + i, s_max=128)
        k = min(r1[i].n_sigma, len(orc.sigma))
        if r1[i].final_s == orc.final_s:
            assert np.max(np.abs(s1[i, :k] - orc.sigma[:k])) <= SIGMA_TOL * orc.sigma[0]
        assert _decision_ok(r1[i], s1[i], Ah, 1e-6, 77 + i), (i, r1[i].rank, orc.rank, r1[i].final_s, orc.final_s)


def test_batched_matches_single_matrix_path(h):
    specs = [(1500, 700, 33), (700, 1500, 60), (800, 800, 9)]
    blocks = []
    for i, (m, n, r) in enumerate(specs):
        A = wl.haar_matrix(m, n, wl.spectrum("step", min(m, n), rank=r, tail_scale=1e-9), seed=40 + i)
        blocks.append(A.to(torch.float32).cuda())
    res, sig = rk.re_rank_estimate_batched(h, blocks, 1e-4, rk.RE_GAUSSIAN, 5, sigma_cap=128)
    for i, B in enumerate(blocks):
        one, s1 = rk.re_rank_estimate(h, B, 1e-4, rk.RE_GAUSSIAN, 5 + i)
        assert one.rank == res[i].rank == specs[i][2] and one.final_s == res[i].final_s
        k = min(len(s1), res[i].n_sigma)
        assert np.max(np.abs(s1[:k] - sig[i, :k])) <= SIGMA_TOL * s1[0]


def test_batched_invalid_block_reported(h):
    good = wl.haar_matrix(400, 300, wl.spectrum("step", 300, rank=7, tail_scale=1e-9), seed=1).to(torch.float32).cuda()
    arr = (rk.re_block * 2)()
    arr[0].ptr, arr[0].m, arr[0].n, arr[0].ld = good.data_ptr(), 400, 300, 300
    arr[1].ptr, arr[1].m, arr[1].n, arr[1].ld = good.data_ptr(), 400, 300, 100       # ld < n
    out = (rk.re_result * 2)()
    rc = rk.lib().re_rank_estimate_batched(h, arr, 2, rk.RE_F32, 1e-4, rk.RE_GAUSSIAN, 3, None, 0, out, None)
    assert rc == 0
    assert out[0].status == 0 and out[0].rank == 7
    assert out[1].status == rk.RE_ERR_ARG


def _points(shapes, seed0):
    out = []
    for i, (m, n) in enumerate(shapes):
        x, y = wl.kernel_points(m, n, seed=seed0 + i)
        out.append((x.float().contiguous().cuda(), y.float().contiguous().cuda()))
    return out


def _dense(x, y):
    """The block of the FP32 points in FP64 (what the oracle sketches)."""
    xd, yd = x.double().cpu().numpy(), y.double().cpu().numpy()
    return 1.0 / np.sqrt(((xd[:, None, :] - yd[None, :, :]) ** 2).sum(axis=2))


def test_matrix_free_kernel_blocks():
    """Matrix-free kernel blocks (entries 1/|x_i - y_j| computed in FP32 as the
    tensor-core sketch consumes them) against the FP64 oracle on the same points,
    against the stored-matrix batched path, and on graph replay."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hm = rk.re_create(0, rk.make_opts(s_max=128, precision=rk.RE_PREC_BF16X3))
    shapes = wl.kernel_block_sizes(14, seed=21, lo=256, hi=1500) + [(100, 1900), (1900, 70), (333, 333)]
    pts = _points(shapes, 600)
    res, sig = rk.re_rank_estimate_kernel_blocks(hm, pts, 1e-6, 77, sigma_cap=128)
    res2, sig2 = rk.re_rank_estimate_kernel_blocks(hm, pts, 1e-6, 77, sigma_cap=128)     # graph replay
    assert [r.rank for r in res] == [r.rank for r in res2] and np.array_equal(sig, sig2)
    dense = [_dense(x, y) for x, y in pts]
    for i, (m, n) in enumerate(shapes):
        orc = alg.rank_estimate(dense[i], 1e-6, kind=alg.GAUSSIAN, seed=77 + i, s_max=128)
        assert res[i].status == 0
        assert bool(res[i].flags & rk.RE_TRANSPOSED) == (m < n)
        if res[i].final_s == orc.final_s:
            k = min(res[i].n_sigma, len(orc.sigma))
            assert np.max(np.abs(sig[i, :k] - orc.sigma[:k])) <= SIGMA_TOL * orc.sigma[0]
        assert _decision_ok(res[i], sig[i], dense[i], 1e-6, 77 + i), (i, res[i].rank, orc.rank)
    # the stored blocks (FP64 distances of the same points, rounded to FP32)
    blocks = [torch.from_numpy(D).float().cuda() for D in dense]
    rs, ss = rk.re_rank_estimate_batched(hm, blocks, 1e-6, rk.RE_GAUSSIAN, 77, sigma_cap=128)
    same = sum(int(a.rank == b.rank) for a, b in zip(res, rs))
    assert same >= len(shapes) - 2, same
    for i in range(len(shapes)):
        if res[i].final_s == rs[i].final_s:
            k = min(res[i].n_sigma, rs[i].n_sigma)
            assert np.max(np.abs(sig[i, :k] - ss[i, :k])) <= SIGMA_TOL * ss[i, 0]
    rk.re_destroy(hm)


def test_matrix_free_errors():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    pts = _points([(300, 200), (256, 260)], 900)
    # coincident points: an infinite entry, reported in that block's status only
    x, y = pts[1]
    y[5] = x[3]
    h32 = rk.re_create(0, rk.make_opts(s_max=128, precision=rk.RE_PREC_FP32))
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate_kernel_blocks(h32, pts, 1e-6, 1)
    assert e.value.code == rk.RE_ERR_UNSUPPORTED
    rk.re_destroy(h32)
    hm = rk.re_create(0, rk.make_opts(s_max=128, precision=rk.RE_PREC_BF16X3))
    res, _ = rk.re_rank_estimate_kernel_blocks(hm, pts, 1e-6, 1)
    assert res[0].status == 0 and res[1].status == rk.RE_ERR_NONFINITE
    rk.re_destroy(hm)


def test_batched_first_pass_autotune_same_bits():
    """The tensor-core ladder's first-pass width (the autotuned N tile of the first
    pass) changes only the number of passes: ranks, widths and sketched values are
    the same bits for every candidate, and the autotuned handle returns them too."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    shapes = wl.kernel_block_sizes(20, seed=41, lo=256, hi=1500) + [(300, 900), (1024, 1024)]
    blocks = [wl.kernel_block(m, n, seed=700 + i).cuda() for i, (m, n) in enumerate(shapes)]
    ref = None
    for w1 in (8, 16, 32, 64, 0):
        hd = rk.re_create(0, rk.make_opts(s_max=128, precision=rk.RE_PREC_BF16X3, batch_first_width=w1))
        try:
            res, sig = rk.re_rank_estimate_batched(hd, blocks, 1e-6, rk.RE_GAUSSIAN, 31, sigma_cap=128)
        finally:
            rk.re_destroy(hd)
        got = ([r.rank for r in res], [r.final_s for r in res], sig)
        if ref is None:
            ref = got
        assert got[0] == ref[0] and got[1] == ref[1] and np.array_equal(got[2], ref[2]), w1
        if w1:
            for r in res:
                assert r.passes == 1 + sum(1 for t in (16, 32, 64, 128) if 2 * w1 <= t <= r.final_s)
