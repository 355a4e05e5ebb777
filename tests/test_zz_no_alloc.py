"""The allocation-free sketch step (re_sketch_apply_noalloc) against the
handle-based re_sketch_apply, through the C ABI.

Callers that may not allocate device memory (stream capture, externally owned
memory pools, real-time paths) use the allocation-free entry point; its output
must equal the regular entry point's.  Two appending calls in a row check that
the shared static scratch carries nothing over from one call to the next.
This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from paper_2105_07388_gb300 import rankest as rk

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hd = rk.re_create(0)
    yield hd
    rk.re_destroy(hd)


@pytest.mark.parametrize("m,n", [(3000, 1000), (700, 2100)])
def test_noalloc_matches_sketch_apply_two_calls(h, m, n):
    A = torch.from_numpy(np.random.default_rng(m).standard_normal((m, n)).astype(np.float32)).cuda()
    rows = max(m, n)
    ax_ref = torch.zeros(rows, 32, device="cuda")
    core_ref = torch.zeros(64, 32, dtype=torch.float64, device="cuda")
    ax_new = torch.zeros(rows, 32, device="cuda")
    core_new = torch.zeros(64, 32, dtype=torch.float64, device="cuda")
    for col0 in (0, 16):                      # two calls in a row, appending
        rk.re_sketch_apply(h, A, col0, 16, rk.RE_GAUSSIAN, 77, ax_ref, core_ref)
        rk.re_sketch_apply_noalloc(A, col0, 16, 77, ax_new, core_new)
        torch.cuda.synchronize()
        c1 = col0 + 16
        a_ref = ax_ref[:, :c1].double().cpu().numpy()
        a_new = ax_new[:, :c1].double().cpu().numpy()
        # the same kernels run on the same inputs: the FP32 tolerance of the
        # parity tests (relative to |A||X|, bounded here by max |AX|) is generous
        tol = 2.0 * (min(m, n) / 32 + 32) * U32 * np.abs(a_ref).max()
        assert np.max(np.abs(a_new - a_ref)) <= tol
        k_ref = core_ref[:2 * c1, :c1].cpu().numpy()
        k_new = core_new[:2 * c1, :c1].cpu().numpy()
        assert np.max(np.abs(k_new - k_ref)) <= 1e-5 * np.abs(k_ref).max()
        # and against the FP64 oracle's core entry by entry, with the FP32 bound of
        # the other core tests (A X and Y (A X) both accumulated in FP32)
        A64 = A.double().cpu().numpy()
        Ao = A64.T if m < n else A64
        X, Y = alg.embeddings(alg.GAUSSIAN, Ao.shape[1], Ao.shape[0], c1, 77)
        ref = Y @ (Ao @ X)
        bound = 4.0 * (Ao.shape[0] / 32 + Ao.shape[1] / 32 + 64) * U32 * (np.abs(Y) @ np.abs(Ao) @ np.abs(X))
        assert np.all(np.abs(k_new - ref) <= bound), float(np.max(np.abs(k_new - ref) / bound))


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    A = torch.zeros(8192, 8192, device="cuda")
    AX = torch.zeros(8192, 1024, device="cuda")
    with pytest.raises(rk.RankEstError) as e:
        rk.re_sketch_apply_noalloc(A, 0, 1024, 1, AX)       # 8192 x 1024 X > 4 Mi floats
    assert e.value.code == rk.RE_ERR_ARG
