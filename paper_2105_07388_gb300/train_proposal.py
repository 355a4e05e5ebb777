"""Train the sketch-size proposal network on the GPU and write proposal.remlp.

Training pairs come from this library itself: for seeded synthetic matrices
with the paper's spectrum families (Sec. 6: exponential, algebraic and step
gaps, here also with a noise floor), the features are those of the s = 16
first sketch (re_mlp_features) and the label is the width class of the plain
doubling ladder's final width (re_rank_estimate).  The matrices are diagonal
(padded with zero rows when m > n); for Gaussian embeddings the sketched
singular values of U diag(sigma) V^T have the same distribution as those of
diag(sigma) (orthogonal invariance of the Gaussian), so this covers every
matrix with these spectra.  The network is trained by the library's own
forward/backward/Adam kernels (re_mlp_train).

    python -m paper_2105_07388_gb300.train_proposal --samples 12000 --out <path>
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2105_07388_gb300 import build, rankest as rk  # noqa: E402


def spectrum(rng, n):
    fam = rng.integers(0, 4)
    i = np.arange(1, n + 1, dtype=np.float64)
    if fam == 0:
        s = 10.0 ** (-rng.uniform(0.002, 0.4) * (i - 1))
    elif fam == 1:
        s = i ** -rng.uniform(0.5, 3.0)
    elif fam == 2:
        r = int(rng.integers(1, 420))
        s = np.where(i <= r, 10.0 ** (-rng.uniform(0, 2) * (i - 1) / max(r, 1)), 0.0)
        s[r:] = 10.0 ** -rng.uniform(5, 12) / i[r:]
    else:
        s = 10.0 ** (-rng.uniform(0.005, 0.1) * (i - 1))
    if rng.random() < 0.4:
        s = np.maximum(s, 10.0 ** -rng.uniform(5, 12))
    return np.sort(s)[::-1] / s.max()


def make_pairs(h, count, seed, sizes):
    rng = np.random.default_rng(seed)
    X = np.zeros((count, 18), dtype=np.float32)
    y = np.zeros(count, dtype=np.int32)
    passes = np.zeros(count, dtype=np.int32)
    bufs = {}
    for t in range(count):
        n = int(rng.choice(sizes))
        m = int(n * rng.choice([1, 2, 4, 8]))
        key = (m, n)
        if key not in bufs:
            if len(bufs) > 6:
                bufs.clear()
                torch.cuda.empty_cache()
            bufs[key] = torch.zeros(m, n, dtype=torch.float32, device="cuda")
        A = bufs[key]
        s = spectrum(rng, n)
        A.diagonal().copy_(torch.from_numpy(s.astype(np.float32)))
        eps = float(10.0 ** -rng.uniform(1.5, 7))
        sk = int(rng.integers(0, 2 ** 31))
        X[t] = rk.re_mlp_features(h, A, eps, sk)
        res, _ = rk.re_rank_estimate(h, A, eps, rk.RE_GAUSSIAN, sk, sigma_cap=0)
        y[t] = int(np.log2(res.final_s // 8))
        passes[t] = res.passes
    return X, y, passes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=12000)
    ap.add_argument("--heldout", type=int, default=1500)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--out", default=os.path.join(HERE, "proposal.remlp"))
    ap.add_argument("--report", default=None)
    a = ap.parse_args()
    build.build()
    h = rk.re_create(0)
    t0 = time.time()
    Xtr, ytr, _ = make_pairs(h, a.samples, 1, [512, 1024, 2048, 4096])
    Xte, yte, pte = make_pairs(h, a.heldout, 2, [1024, 2048, 4096])
    t_data = time.time() - t0
    rk.re_mlp_init(h, 7)
    losses = rk.re_mlp_train(h, Xtr, ytr, epochs=a.epochs, batch=256, lr=2e-3, weight_decay=1e-5, seed=3)
    cls, _ = rk.re_mlp_predict(h, Xte)
    rk.re_mlp_save(h, a.out)
    # passes over A on the held-out set: plain ladder vs proposal (same answers by construction)
    over = cls >= yte
    learned_passes = np.where(yte <= 1, pte, np.where(over, 2, 2 + (yte - np.maximum(cls, 2))))
    rep = {"train_samples": int(a.samples), "heldout": int(a.heldout), "data_seconds": t_data,
           "final_loss": float(losses[-1]), "first_loss": float(losses[0]),
           "heldout_exact_class": float(np.mean(cls == yte)),
           "heldout_at_or_above": float(np.mean(over)),
           "plain_mean_passes": float(np.mean(pte)), "learned_mean_passes_est": float(np.mean(learned_passes)),
           "label_histogram": np.bincount(ytr, minlength=12).tolist()}
    print(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    rk.re_destroy(h)


if __name__ == "__main__":
    main()
