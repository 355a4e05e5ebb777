"""Proposal network kernels against the FP64 reference, and the learned
estimator against the plain one (identical answers by the nested-prefix
property of appended sketches)."""
import os

import numpy as np
import pytest
import torch

from oracle import algorithm1 as alg
from oracle import mlp
from paper_2105_07388_gb300 import rankest as rk
from paper_2105_07388_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(rk.__file__), "proposal.remlp")


@pytest.fixture(scope="module")
def h():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2105_07388_gb300 import build
    build.build()
    hd = rk.re_create(0)
    yield hd
    rk.re_destroy(hd)


def _params(seed):
    return (np.random.default_rng(seed).standard_normal(mlp.NPARAMS) * 0.15).astype(np.float32)


def test_forward_matches_oracle(h):
    p = _params(1)
    rk.re_mlp_set_params(h, p)
    X = np.random.default_rng(2).standard_normal((300, 18)).astype(np.float32)
    cls, logits = rk.re_mlp_predict(h, X)
    z, _, _ = mlp.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(logits - z)) <= 1e-4 * np.max(np.abs(z)) + 1e-5
    assert np.mean(cls == np.argmax(z, axis=1)) > 0.99


def test_gradient_matches_oracle(h):
    p = _params(3)
    rk.re_mlp_set_params(h, p)
    rng = np.random.default_rng(4)
    X = rng.standard_normal((257, 18)).astype(np.float32)
    y = rng.integers(0, 12, 257).astype(np.int32)
    loss, g = rk.re_mlp_grad(h, X, y)
    lref, gref = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y)
    assert abs(loss - lref) <= 1e-4 * abs(lref)
    # FP32 accumulation (atomics over 257 samples) against FP64
    assert np.max(np.abs(g - gref)) <= 1e-4 * np.max(np.abs(gref)) + 1e-7
    rel = np.linalg.norm(g - gref) / np.linalg.norm(gref)
    assert rel < 1e-5


def test_training_reduces_loss_and_checkpoint_resumes(h, tmp_path):
    rk.re_mlp_init(h, 11)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2048, 18)).astype(np.float32)
    y = (np.clip((X[:, 0] * 2 + 6), 0, 11)).astype(np.int32)       # learnable labels
    losses = rk.re_mlp_train(h, X, y, epochs=8, batch=128, lr=3e-3, seed=1)
    assert losses[-1] < 0.5 * losses[0]
    path = str(tmp_path / "net.remlp")
    rk.re_mlp_save(h, path)
    p1 = rk.re_mlp_get_params(h)
    h2 = rk.re_create(0)
    try:
        rk.re_mlp_load(h2, path)
        assert np.array_equal(rk.re_mlp_get_params(h2), p1)
        # resuming continues from the saved Adam state: one more epoch on both handles
        l1 = rk.re_mlp_train(h, X, y, epochs=1, batch=128, lr=3e-3, seed=9)
        l2 = rk.re_mlp_train(h2, X, y, epochs=1, batch=128, lr=3e-3, seed=9)
        # per-sample gradients are accumulated with FP32 atomics, so the two runs
        # agree to rounding level (summation order differs), not bit for bit
        assert np.allclose(rk.re_mlp_get_params(h), rk.re_mlp_get_params(h2), rtol=1e-3, atol=1e-4)
        assert abs(l1[0] - l2[0]) < 1e-3
    finally:
        rk.re_destroy(h2)


def test_features_match_oracle(h):
    sig = wl.spectrum("fp", 600)
    A = wl.haar_matrix(900, 600, sig, seed=2).to(torch.float32)
    f = rk.re_mlp_features(h, A.cuda(), 1e-4, 31)
    s16 = alg.sketched_sigma(A.double().numpy(), 16, alg.GAUSSIAN, 31)
    ref = mlp.features(s16, 1e-4, 900, 600)
    assert np.max(np.abs(f - ref)) < 1e-3


@pytest.mark.parametrize("m,n,rank", [(1200, 600, 5), (1500, 1000, 60), (2048, 1024, 150), (900, 2000, 30)])
def test_learned_equals_plain(h, m, n, rank):
    # any network gives the plain answer: the nested leading blocks are checked in ladder order
    rk.re_mlp_init(h, 5)
    A = wl.haar_matrix(m, n, wl.spectrum("step", min(m, n), rank=rank, tail_scale=1e-9), seed=m).to(torch.float32).cuda()
    plain, sp = rk.re_rank_estimate(h, A, 1e-4, rk.RE_GAUSSIAN, 3)
    rk.re_set_opts(h, rk.make_opts(learned=1))
    try:
        learned, sl = rk.re_rank_estimate(h, A, 1e-4, rk.RE_GAUSSIAN, 3)
    finally:
        rk.re_set_opts(h, rk.re_opts_default())
    assert learned.rank == plain.rank == rank and learned.final_s == plain.final_s
    assert np.max(np.abs(sl - sp)) <= 1e-4 * sp[0]


def test_trained_network_saves_passes(h):
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained proposal network in the package")
    rk.re_mlp_load(h, WEIGHTS)
    rng = np.random.default_rng(2024)
    plain_passes, learned_passes = [], []
    for t in range(12):
        n = int(rng.choice([512, 1024, 2048]))
        m = 2 * n
        fam = ["se", "fp", "step", "sp"][t % 4]
        sig = wl.spectrum(fam, n, rank=int(rng.integers(20, 220)), tail_scale=1e-9) if fam == "step" else wl.spectrum(fam, n)
        A = wl.haar_matrix(m, n, sig, seed=1000 + t).to(torch.float32).cuda()
        eps = float(10.0 ** -rng.uniform(2, 6))
        plain, _ = rk.re_rank_estimate(h, A, eps, rk.RE_GAUSSIAN, 77 + t)
        rk.re_set_opts(h, rk.make_opts(learned=1))
        try:
            learned, _ = rk.re_rank_estimate(h, A, eps, rk.RE_GAUSSIAN, 77 + t)
        finally:
            rk.re_set_opts(h, rk.re_opts_default())
        assert learned.rank == plain.rank and learned.final_s == plain.final_s
        plain_passes.append(plain.passes)
        learned_passes.append(learned.passes)
    assert np.mean(learned_passes) < np.mean(plain_passes)
