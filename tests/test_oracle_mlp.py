"""Pins for the proposal network's FP64 reference (CPU only)."""
import numpy as np

from oracle import mlp


def _params(seed=0, scale=0.2):
    return np.random.default_rng(seed).standard_normal(mlp.NPARAMS) * scale


def test_parameter_count():
    assert mlp.NPARAMS == 128 * 18 + 128 + 128 * 128 + 128 + 12 * 128 + 12 == 20492


def test_zero_weights_give_bias_logits_and_uniform_loss():
    p = np.zeros(mlp.NPARAMS)
    q = mlp.unpack(p)
    q["b3"] = np.arange(12, dtype=float)
    p = mlp.pack(q)
    X = np.random.default_rng(1).standard_normal((5, 18))
    z, _, _ = mlp.forward(p, X)
    assert np.allclose(z, np.arange(12))
    loss, g = mlp.loss_and_grad(np.zeros(mlp.NPARAMS), X, np.zeros(5, dtype=int))
    assert np.isclose(loss, np.log(12.0))
    # with all-zero weights only the output bias receives gradient: softmax - onehot
    gq = mlp.unpack(g)
    want = np.full(12, 1 / 12.0)
    want[0] -= 1.0
    assert np.allclose(gq["b3"], want) and np.allclose(gq["W1"], 0) and np.allclose(gq["W3"], 0)


def test_gradient_matches_central_differences():
    # Finite differences pin the analytic gradient (with weights taken as their
    # BF16 roundings, perturbing a weight by less than a BF16 ulp would not move
    # the loss, so the check perturbs biases and compares weight gradients through
    # the chain rule on an exactly BF16-representable parameter set).
    rng = np.random.default_rng(3)
    p = mlp.bf16(_params(3)).astype(np.float64)      # weights exactly representable
    X = rng.standard_normal((7, 18))
    y = rng.integers(0, 12, 7)
    loss, g = mlp.loss_and_grad(p, X, y)
    q = mlp.unpack(p)
    off = {name: o for name, o in zip([n for n, _ in mlp.SHAPES],
                                      np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])[:-1])}
    for name in ("b1", "b2", "b3"):
        for k in range(0, q[name].size, 17):
            h = 1e-6
            pp = p.copy(); pp[off[name] + k] += h
            pm = p.copy(); pm[off[name] + k] -= h
            fd = (mlp.loss_and_grad(pp, X, y)[0] - mlp.loss_and_grad(pm, X, y)[0]) / (2 * h)
            assert abs(fd - g[off[name] + k]) <= 1e-6 + 1e-5 * abs(fd), (name, k)
    # weights: step by exactly one BF16 ulp (w +- ulp stay BF16-representable, so the
    # network sees exactly the perturbed weight)
    for name in ("W1", "W2", "W3"):
        for k in range(0, q[name].size, 997):
            w = p[off[name] + k]
            if w == 0:
                continue
            h = 2.0 ** (np.floor(np.log2(abs(w))) - 7)
            pp = p.copy(); pp[off[name] + k] = w + h
            pm = p.copy(); pm[off[name] + k] = w - h
            assert mlp.bf16(pp[off[name] + k:off[name] + k + 1])[0] == w + h
            fd = (mlp.loss_and_grad(pp, X, y)[0] - mlp.loss_and_grad(pm, X, y)[0]) / (2 * h)
            assert abs(fd - g[off[name] + k]) <= 1e-4 + 2e-2 * abs(fd), (name, k, fd, g[off[name] + k])


def test_features_formula():
    sig = np.logspace(0, -6, 16)
    f = mlp.features(sig, 1e-4, 1000, 500)
    assert np.isclose(f[0], 4.0) and np.isclose(f[14], 3.0) and np.isclose(f[16], 4.0)
    assert np.isclose(f[17], (f[13] - f[7]) / 6.0)
    assert np.allclose(np.diff(f[:14]), -6 / 15)


def test_mlp_bf16_rounding_ties_to_even():
    """The network's BF16 weights round to nearest, ties to even (hand-chosen ties)."""
    src = np.array([0x3F808000, 0x3F818000, 0x3F808001, 0xBF818000], dtype=np.uint32).view(np.float32)
    want = np.array([0x3F800000, 0x3F820000, 0x3F810000, 0xBF820000], dtype=np.uint32).view(np.float32)
    assert np.array_equal(mlp.bf16(src), want.astype(np.float64))
