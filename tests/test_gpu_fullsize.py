"""Parity at the headline workload's full size: the 65536 x 16384 FP32 matrix
(sigma_i = 1 for i <= 200, then 1e-6 / i; eps = 1e-4; true rank 200), on the
BF16x3 tensor-core path in the launch configuration bench.py times (the doubling
ladder's appends of 8, 8, 16, 32, 64 and 128 columns).

The oracle cannot sketch the whole matrix in seconds, so it checks sampled
outputs one by one: entries of AX (rows of A times oracle X columns), entries of
the core (oracle Y rows times oracle AX columns over all 65536 rows), and the
estimate against what the construction fixes (rank 200 at s = 256, the 200 unit
singular values sketched inside the Gaussian embedding's range, the next one at
the 1e-6 level).

The structured embeddings the benchmark also times at this size get the same
sampled checks, in the estimator's launch configuration under BF16x3: the SRHT's
appended +-1 columns (s up to 128), the HRTT's and the hashed randomized DCT's
whole width-256 sketches (one and three BF16 planes of X), and the core of the
SRCT left embedding on the Gaussian A X, with the estimates of the hashed and
SRCT forms against the construction."""
import numpy as np
import pytest
import torch

import bench
from oracle import algorithm1 as alg
from oracle import rng
from paper_2105_07388_gb300 import rankest as rk

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24
W = bench.WORKLOADS["large"]
SEED = W["sketch_seed"]
APPENDS = [(0, 8), (8, 8), (16, 16), (32, 32), (64, 64), (128, 128)]


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    A = bench.build_matrix(W, "cuda")
    m, n = A.shape
    h = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    AX = torch.zeros(m, 256, dtype=torch.float32, device="cuda")
    core = torch.zeros(512, 256, dtype=torch.float64, device="cuda")
    for c0, cnt in APPENDS:
        rk.re_sketch_apply(h, A, c0, cnt, rk.RE_GAUSSIAN, SEED, AX, core)
    res, sig = rk.re_rank_estimate(h, A, W["eps"], rk.RE_GAUSSIAN, SEED)
    torch.cuda.synchronize()
    out = {"A_host": A.cpu().numpy(), "AX": AX.cpu().numpy(), "core": core.cpu().numpy(),
           "res": res, "sig": sig}
    # SRHT: the ladder's appends up to 128 columns; HRTT and HRCT: the width-256
    # sketch the estimator forms from column 0
    for c0, cnt in APPENDS[:-1]:
        rk.re_sketch_apply(h, A, c0, cnt, rk.RE_SRHT, SEED, AX)
    out["AX_srht"] = AX[:, :128].cpu().numpy()
    for kind, key in ((rk.RE_HRTT, "AX_hrtt"), (rk.RE_HRCT, "AX_hrct")):
        AX.zero_()
        rk.re_sketch_apply(h, A, 0, 256, kind, SEED, AX)
        out[key] = AX.cpu().numpy()
        out["res_" + key[3:]], _ = rk.re_rank_estimate(h, A, W["eps"], kind, SEED)
    rk.re_destroy(h)
    # SRCT left embedding on the Gaussian A X (the bench's srct_y variant)
    hs = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3, y_kind=rk.RE_SRCT))
    core.zero_()
    for c0, cnt in APPENDS:
        rk.re_sketch_apply(hs, A, c0, cnt, rk.RE_GAUSSIAN, SEED, AX, core)
    out["core_srct"] = core.cpu().numpy()
    out["res_srct"], _ = rk.re_rank_estimate(hs, A, W["eps"], rk.RE_GAUSSIAN, SEED)
    rk.re_destroy(hs)
    torch.cuda.synchronize()
    del A, AX, core
    torch.cuda.empty_cache()
    return out


def test_sampled_ax_entries(full):
    A_host, AX = full["A_host"], full["AX"]
    m, n = A_host.shape
    gen = np.random.default_rng(2)
    rows = np.sort(gen.choice(m, 24, replace=False))
    rows[-1] = m - 1                                     # the ragged last row tile
    A64 = A_host[rows].astype(np.float64)
    for c0, cnt in APPENDS:
        X = rng.gaussian_x(n, cnt, SEED, col0=c0)
        ref = A64 @ X
        bound = 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
        err = np.abs(AX[rows, c0:c0 + cnt].astype(np.float64) - ref)
        assert np.all(err <= bound), (c0, float(np.max(err / bound)))


def _sample_rows(m):
    gen = np.random.default_rng(2)
    rows = np.sort(gen.choice(m, 24, replace=False))
    rows[-1] = m - 1                                     # the ragged last row tile
    return rows


def test_sampled_ax_entries_srht(full):
    """The SRHT's appended +-1 columns (D H S^T, exact in BF16) through the
    tensor-core contraction: the Gaussian sketch's bound."""
    A_host, AX = full["A_host"], full["AX_srht"]
    m, n = A_host.shape
    rows = _sample_rows(m)
    A64 = A_host[rows].astype(np.float64)
    X = rng.srtt_x(n, 128, SEED)
    bound = 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
    err = np.abs(AX[rows].astype(np.float64) - A64 @ X)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_sampled_ax_entries_hrtt(full):
    """The HRTT's width-256 X (integer entries up to the bucket size 64, one exact
    BF16 plane): the Gaussian sketch's bound."""
    A_host, AX = full["A_host"], full["AX_hrtt"]
    m, n = A_host.shape
    rows = _sample_rows(m)
    A64 = A_host[rows].astype(np.float64)
    X = rng.hrtt_x(n, 256, SEED)
    bound = 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
    err = np.abs(AX[rows].astype(np.float64) - A64 @ X)
    assert np.all(err <= bound), float(np.max(err / bound))


def test_sampled_ax_entries_hrct(full):
    """The hashed randomized DCT's width-256 X: FP32 entries (a compensated sum of
    the bucket's 64 table cosines, within 2u |x| + 4 sqrt(2) u L of the exact value)
    as three BF16 planes, then the Gaussian sketch's accumulation bound."""
    A_host, AX = full["A_host"], full["AX_hrct"]
    m, n = A_host.shape
    rows = _sample_rows(m)
    A64 = A_host[rows].astype(np.float64)
    X = rng.hrct_x(n, 256, SEED)
    L = n // 256
    xerr = 2.0 * U32 * np.abs(X) + 4.0 * U32 * np.sqrt(2.0) * L
    bound = np.abs(A64) @ xerr + 2.0 * (n / 16 + 32) * U32 * (np.abs(A64) @ np.abs(X)) + 1e-35
    err = np.abs(AX[rows].astype(np.float64) - A64 @ X)
    assert np.all(err <= bound), float(np.max(err / bound))


def _oracle_ax_columns(A_host, cols):
    """Oracle A X columns (and |A| |X|) over all rows, for Gaussian X columns `cols`."""
    m, n = A_host.shape
    X = np.concatenate([rng.gaussian_x(n, 1, SEED, col0=c) for c in cols], axis=1)
    axc = np.zeros((m, len(cols)))
    axa = np.zeros((m, len(cols)))
    for r0 in range(0, m, 8192):
        blk = A_host[r0:r0 + 8192].astype(np.float64)
        axc[r0:r0 + 8192] = blk @ X
        axa[r0:r0 + 8192] = np.abs(blk) @ np.abs(X)
    return axc, axa


def test_sampled_core_entries_srct(full):
    """The SRCT left embedding (DCT-II rows of the sampled frequencies, three BF16
    planes on the tensor cores) on the Gaussian A X: sampled core entries against
    the oracle's Y row times the oracle's A X column over all 65536 rows."""
    A_host, core = full["A_host"], full["core_srct"]
    m, n = A_host.shape
    picks = [(3, 5), (40, 21), (300, 140), (511, 255)]
    cols = sorted({c for _, c in picks})
    axc, axa = _oracle_ax_columns(A_host, cols)
    for q, c in picks:
        y = rng.srct_y(1, m, SEED, row0=q)[0]
        j = cols.index(c)
        ref = y @ axc[:, j]
        bound = 4.0 * (m / 32 + n / 32 + 64) * U32 * (np.abs(y) @ axa[:, j])
        assert abs(core[q, c] - ref) <= bound, (q, c, core[q, c], ref, bound)


def test_structured_estimates_fixed_by_construction(full):
    """HRTT and HRCT X (Gaussian Y) and Gaussian X with SRCT Y: the hashing and the
    DCT keep the embedding on this coherent matrix, so each returns rank 200 at
    s = 256 with the gap at 200, as the Gaussian sketch does."""
    for key in ("res_hrtt", "res_hrct", "res_srct"):
        r = full[key]
        assert (r.status, r.rank, r.final_s, r.gap_index) == (0, 200, 256, 200), key
        assert r.flags & rk.RE_CONVERGED


def test_sampled_core_entries(full):
    A_host, core = full["A_host"], full["core"]
    m, n = A_host.shape
    # (row q, column c) of the 512 x 256 core, from blocks appended at different widths
    picks = [(3, 5), (40, 21), (300, 140), (511, 255)]
    cols = sorted({c for _, c in picks})
    X = np.concatenate([rng.gaussian_x(n, 1, SEED, col0=c) for c in cols], axis=1)
    axc = np.zeros((m, len(cols)))
    axa = np.zeros((m, len(cols)))
    for r0 in range(0, m, 8192):                        # oracle AX columns over all rows
        blk = A_host[r0:r0 + 8192].astype(np.float64)
        axc[r0:r0 + 8192] = blk @ X
        axa[r0:r0 + 8192] = np.abs(blk) @ np.abs(X)
    for q, c in picks:
        y = rng.gaussian_y(1, m, SEED, row0=q)[0]
        j = cols.index(c)
        ref = y @ axc[:, j]
        bound = 4.0 * (m / 32 + n / 32 + 64) * U32 * (np.abs(y) @ axa[:, j])
        assert abs(core[q, c] - ref) <= bound, (q, c, core[q, c], ref, bound)


def test_estimate_fixed_by_construction(full):
    res, sig = full["res"], full["sig"]
    assert res.status == 0 and res.rank == 200 and res.final_s == 256 and res.passes == 6
    assert res.flags & rk.RE_CONVERGED
    # the 200 unit singular values: sigma^ are those of (Y U)(V^T X) / sqrt(s r2),
    # a 512 x 200 times a 200 x 256 Gaussian product, whose extreme singular
    # values sit near the products of the Marchenko-Pastur edges
    # (1 -+ sqrt(200/256)) (1 -+ sqrt(200/512)) = 0.044 .. 3.06; factor 2 margins.
    # The tail (1e-6 / i) stays near the FP32 floor, far below eps.
    lo = (1 - np.sqrt(200 / 256)) * (1 - np.sqrt(200 / 512))
    hi = (1 + np.sqrt(200 / 256)) * (1 + np.sqrt(200 / 512))
    assert np.all(sig[:200] > lo / 2) and np.all(sig[:200] < 2 * hi)
    assert sig[200] <= 1e-4 * sig[0]
    assert res.gap_index == 200
