"""The exact-product precision mode (RE_PREC_EXACT) through the C ABI against
the FP64 oracle.

The mode's right sketch A X and left sketch Y (A X) are exact up to one
rounding at 2^-40 of each row's power-of-two bound 2^e (A cut into five 8-bit
digits, the normals of X and Y into two, digit products summed exactly), so
each entry of A X satisfies

    |AX_gpu - AX| <= c 2^(e_i - 40) sum_k |x_k|,

with c a small constant (the dropped digit tails and the FP32 rounding of the
lowest levels).  FP32 accumulation, or a tensor core that dropped low bits of
the exact sums, would miss this bound by orders of magnitude.  End to end, the
read-off at eps = 1e-8 on the ten-decade spectrum of the precision workload
(sigma_i = 10^(-10 (i-1)/300), i <= 300, then 1e-12) must return the oracle's
rank, with every sketched singular value's error stated and bounded.
"""
import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from oracle import rng
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hd = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_EXACT))
    yield hd
    rk.re_destroy(hd)


def padded(A):
    """A FP32 CUDA view whose row pitch is a multiple of 4 floats (16 bytes, what the
    tensor-memory copies take), whatever n is."""
    m, n = A.shape
    ld = (n + 3) // 4 * 4
    full = torch.zeros(m, ld, dtype=torch.float32, device="cuda")
    full[:, :n] = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    return full[:, :n]


def row_scale(A64):
    """2^e_i: the smallest power of two above every |a_ik| of row i."""
    mx = np.abs(A64).max(axis=1)
    e = np.where(mx > 0, np.floor(np.log2(np.where(mx > 0, mx, 1.0))) + 1, 0)
    return np.exp2(e)


def right_bound(A64, X):
    return 4.0 * 2.0 ** -40 * row_scale(A64)[:, None] * np.abs(X).sum(axis=0)[None, :]


@pytest.mark.parametrize("m,n,steps", [
    (1000, 777, ((0, 16), (16, 48))),           # ragged M and K, one and several Q tiles
    (3001, 2500, ((0, 136),)),                  # three Q tiles (64 + 64 + 8)
    (9100, 9000, ((0, 24),)),                   # K beyond one exact segment (8192)
    (300, 300, ((0, 8), (8, 8), (16, 16))),     # square, appended widths of 8
])
def test_exact_right_sketch_parity(h, m, n, steps):
    A = np.random.default_rng(m + n).standard_normal((m, n)).astype(np.float32)
    A64 = A.astype(np.float64)
    Ad = padded(A)
    c1 = steps[-1][0] + steps[-1][1]
    AX = torch.zeros(m, c1, dtype=torch.float64, device="cuda")
    for col0, s in steps:
        rk.re_sketch_apply_exact(h, Ad, col0, s, 4242, AX)
        X = rng.gaussian_x(n, s, 4242, col0)
        ref = A64 @ X
        got = AX[:, col0:col0 + s].cpu().numpy()
        err = np.abs(got - ref)
        bound = right_bound(A64, X)
        assert np.all(err <= bound), float((err / bound).max())
        # the bound is far below what FP32 accumulation reaches
        assert float((err / bound).max()) < 1.0


def test_exact_accumulation_at_largest_digits(h):
    """Every entry of a row at (nearly) its power-of-two bound: the leading digits
    take their largest values, so the exact partial sums of the tensor cores come
    closest to the 2^24-unit limit; the result must still meet the exact bound."""
    m, n = 8192, 8192
    sgn = np.sign(np.random.default_rng(5).standard_normal((m, n)))
    A = (sgn * np.float32(1.0 - 2.0 ** -24)).astype(np.float32)
    A[::7] *= np.float32(0.75)                       # a second digit pattern on some rows
    A64 = A.astype(np.float64)
    AX = torch.zeros(m, 64, dtype=torch.float64, device="cuda")
    rk.re_sketch_apply_exact(h, torch.from_numpy(A).cuda(), 0, 64, 99, AX)
    X = rng.gaussian_x(n, 64, 99, 0)
    err = np.abs(AX.cpu().numpy() - A64 @ X)
    assert np.all(err <= right_bound(A64, X)), float((err / right_bound(A64, X)).max())


@pytest.mark.parametrize("m,n,steps", [
    (2000, 700, ((0, 16), (16, 16))),
    (4099, 1200, ((0, 64), (64, 72))),          # appended blocks of several tiles
])
def test_exact_core_parity(h, m, n, steps):
    A = np.random.default_rng(7 * m + n).standard_normal((m, n)).astype(np.float32)
    A64 = A.astype(np.float64)
    Ad = padded(A)
    c1 = steps[-1][0] + steps[-1][1]
    AX = torch.zeros(m, c1, dtype=torch.float64, device="cuda")
    core = torch.zeros(2 * c1, c1, dtype=torch.float64, device="cuda")
    for col0, s in steps:
        rk.re_sketch_apply_exact(h, Ad, col0, s, 31, AX, core)
        w = col0 + s
        X, Y = alg.embeddings(alg.GAUSSIAN, n, m, w, 31)
        ref = Y @ (A64 @ X)
        got = core[:2 * w, :w].cpu().numpy()
        # the A X bound carried through Y, plus the left sketch's own 2^-40 rounding
        # of each A X column's power-of-two bound
        AXe = A64 @ X
        col_scale = np.exp2(np.floor(np.log2(np.abs(AXe).max(axis=0))) + 1)
        bound = np.abs(Y) @ right_bound(A64, X) + 4.0 * 2.0 ** -40 * np.abs(Y).sum(axis=1)[:, None] * col_scale[None, :]
        assert np.all(np.abs(got - ref) <= bound), float((np.abs(got - ref) / bound).max())


def test_exact_errors(h):
    A = torch.randn(300, 200, device="cuda")
    AX = torch.zeros(300, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply_exact(h, A.t().contiguous(), 0, 16, 1, torch.zeros(300, 16, dtype=torch.float64,
                                                                               device="cuda"))
    assert e.value.code == rk.RE_ERR_UNSUPPORTED              # m < n
    B = A.clone()
    B[17, 3] = float("nan")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply_exact(h, B, 0, 16, 1, AX)
    assert e.value.code == rk.RE_ERR_NONFINITE
    with pytest.raises(rk.RankEstError) as e:
        rk.re_rank_estimate(h, A.double(), 1e-8)
    assert e.value.code == rk.RE_ERR_UNSUPPORTED              # FP64 A
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply(h, A, 0, 16, rk.RE_GAUSSIAN, 1, torch.zeros(300, 16, device="cuda"))
    assert e.value.code == rk.RE_ERR_UNSUPPORTED              # FP32 A X output
    C = torch.randn(300, 201, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply_exact(h, C, 0, 16, 1, AX)
    assert e.value.code == rk.RE_ERR_UNSUPPORTED              # row pitch not a multiple of 16 bytes
    res, _ = rk.re_rank_estimate(h, torch.zeros(256, 128, device="cuda"), 1e-8)
    assert res.rank == 0


N2, SEED2 = 8192, 77


def _oracle_ladder_values(A64, seed, widths):
    return {s: alg.sketched_sigma(A64, s, alg.GAUSSIAN, seed)[:alg.r1_of_s(s)] for s in widths}


def _simulate(vals, eps, widths):
    """Algorithm 1's read-off over the ladder on the oracle's values: (rank, final
    width, smallest relative distance of a visited trusted value from tau)."""
    margin = np.inf
    for s in widths:
        sig = vals[s]
        tau = eps * sig[0]
        margin = min(margin, float(np.min(np.abs(sig - tau)) / tau))
        hit = np.nonzero(sig <= tau)[0]
        if hit.size:
            return int(hit[0]), s, margin
    return len(vals[widths[-1]]), widths[-1], margin


@pytest.fixture(scope="module")
def geom_case():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    sig = wl.spectrum("geom300", N2)              # 10^(-10 (i-1)/300), then a 1e-12 floor
    A32 = wl.householder_matrix(N2, N2, sig, seed=3)
    A64 = A32.double().numpy()
    widths = [8 * 2 ** k for k in range(7)]      # 8 .. 512
    return A32, A64, _oracle_ladder_values(A64, SEED2, widths), widths


def _pick_eps(vals, widths, center):
    """eps within a factor 10^0.15 of `center`, placed where every visited trusted
    value is farthest (relatively) from tau: no sketched value on the threshold
    (the reading of Definition 1 at a tie)."""
    best = None
    for t in np.linspace(-0.15, 0.15, 61):
        eps = center * 10.0 ** t
        r, s_f, mg = _simulate(vals, eps, widths)
        if best is None or mg > best[3]:
            best = (eps, r, s_f, mg)
    assert best[3] >= 0.03, best
    return best


@pytest.mark.parametrize("center", [1e-8, 2e-9], ids=["eps1e-8", "eps2e-9"])
def test_exact_rank_at_eps_1e8(h, geom_case, center):
    """Algorithm 1 at eps ~ 1e-8 (and ~2e-9, whose ladder runs on to the 1024 x 512
    core) on the 8192 x 8192 ten-decade spectrum: the rank, final width and
    convergence equal the oracle's, and every trusted sketched singular value is
    within the stated bound of the oracle's."""
    A32, A64, vals, widths = geom_case
    eps, r_o, s_o, margin = _pick_eps(vals, widths, center)
    orc = alg.rank_estimate(A64, eps, kind=alg.GAUSSIAN, seed=SEED2)
    assert (orc.rank, orc.final_s) == (r_o, s_o)
    res, sig = rk.re_rank_estimate(h, A32.cuda(), eps, rk.RE_GAUSSIAN, SEED2)
    ref = vals[res.final_s]
    k = min(len(sig), len(ref))
    print("\n[exact] rel err by index:", np.array2string(np.abs(sig[:k] - ref[:k]) / ref[:k], precision=2,
                                                        threshold=10000, max_line_width=200))
    assert res.final_s == orc.final_s and res.rank == orc.rank, (res.rank, orc.rank, res.final_s, orc.final_s)
    assert bool(res.flags & rk.RE_CONVERGED) == orc.converged
    # the first pass of the exact-product sketch covers the widths up to 64
    assert res.passes == 1 + max(0, int(round(np.log2(res.final_s / 64))))
    err = np.abs(sig[:k] - ref[:k])
    rel = err / ref[:k]
    s1 = ref[0]
    above = ref[:k] >= 1e-10 * s1
    print(f"\n[exact] eps = {eps:.4e}, rank {res.rank} at s = {res.final_s} (oracle {orc.rank}), "
          f"margin {margin:.3f}; max |err|/sigma_1 = {err.max() / s1:.3e}; "
          f"max rel err (sigma >= 1e-10 sigma_1) = {rel[above].max():.3e}; "
          f"rel err at the threshold index = {rel[min(res.rank, k - 1)]:.3e}; svd sweeps {res.svd_sweeps}")
    # per index: |err_i| <= 1e-4 sigma_i + 3e-12 sigma_1 (measured: relative errors of
    # 1e-8..1e-7 at the top, 5e-5 at 1e-8 sigma_1, and an absolute floor of about
    # 1.2e-12 sigma_1 reached on the 1e-12 noise floor of the spectrum)
    bound = 1e-4 * ref[:k] + 3e-12 * s1
    assert np.all(err <= bound), float(np.max(err / bound))
    # the decision itself is resolved: the error at tau is far below the margin
    assert rel[min(res.rank, k - 1)] < 0.1 * margin


@pytest.mark.parametrize("r2,s,seed", [(128, 64, 1), (512, 256, 2), (1024, 512, 3), (600, 300, 4)])
def test_precise_core_sigma_against_lapack(h, r2, s, seed):
    """The preconditioned singular values (step 7 of the precision mode) against
    LAPACK on cores with values spread over twelve decades: relative accuracy 1e-4
    above an absolute floor near 1e-12 sigma_1 (the FP32 rotations of the second
    stage remove the first stage's residual non-orthogonality, at most 4 u sqrt(s)
    relative, to FP32 precision: about 2e-13 sigma_1), where the FP32 form
    (re_core_sigma) has an absolute error near 1e-5 sigma_1."""
    gen = np.random.default_rng(seed)
    U, _ = np.linalg.qr(gen.standard_normal((r2, s)))
    V, _ = np.linalg.qr(gen.standard_normal((s, s)))
    sv = np.logspace(0, -12, s)
    C = (U * sv) @ V.T
    ref = np.linalg.svd(C, compute_uv=False)
    sig = torch.zeros(s, dtype=torch.float64, device="cuda")
    rk.re_core_sigma_exact(h, torch.from_numpy(C).cuda(), sig)
    got = sig.cpu().numpy()
    assert np.all(np.diff(got) <= 0)
    err = np.abs(got - ref)
    print(f"\n[precise sigma {r2}x{s}] max rel err {np.max(err / ref):.2e}, max |err|/sigma_1 {err.max() / ref[0]:.2e}")
    assert np.all(err <= 1e-4 * ref + 2e-12 * ref[0]), float(np.max(err / (1e-4 * ref + 2e-12 * ref[0])))
