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
forward/backward/Adam kernels (re_mlp_train).  The held-out evaluation runs
the real dense path: dense matrices with m and n up to 16384, each estimated by
the plain ladder and by the learned ladder, with the passes over A counted.

    python -m paper_2105_07388_gb300.train_proposal --samples 200000 --heldout 10000 \
        --report paper_2105_07388_gb300/proposal_report.json
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2105_07388_gb300 import build, rankest as rk  # noqa: E402


FAMILIES = ("exponential_to_floor", "step_gap", "ten_decades_floor", "kernel_decay", "algebraic",
            "exponential", "graded_step")


def spectrum(rng, n):
    """Seeded singular values (descending, sigma_1 = 1) and the family index.

    The families follow the workloads the estimator is run on: the 2048 x 1024
    matrix's exponential decay to a floor, the 65536 x 16384 matrix's step gap
    with a 1/i tail, the precision workload's ten decades then a noise floor,
    the off-diagonal kernel blocks' fast decay to the FP32 floor (Sec. 6's
    exponential, algebraic and step families); each with its rates, knees and
    floors drawn at random."""
    fam = int(rng.integers(0, len(FAMILIES)))
    i = np.arange(1, n + 1, dtype=np.float64)
    if fam == 0:
        knee = int(rng.integers(5, max(6, min(n, 450))))
        s = 10.0 ** (-rng.uniform(0.03, 0.25) * (i - 1))
        s[knee:] = 10.0 ** -rng.uniform(8, 13)
    elif fam == 1:
        r = int(rng.integers(1, max(2, min(n // 2, 480))))
        s = np.where(i <= r, 1.0, 10.0 ** -rng.uniform(3.5, 9) / i)
    elif fam == 2:
        L = int(rng.integers(30, max(31, min(n, 450))))
        s = np.where(i <= L, 10.0 ** (-rng.uniform(4, 12) * (i - 1) / L), 10.0 ** -rng.uniform(10, 14))
    elif fam == 3:
        s = np.exp(-rng.uniform(0.02, 1.0) * (i - 1) ** rng.uniform(0.5, 1.0))
        s = np.maximum(s, 10.0 ** -rng.uniform(6, 8))
    elif fam == 4:
        s = i ** -rng.uniform(0.5, 3.0)
    elif fam == 5:
        s = 10.0 ** (-rng.uniform(0.002, 0.4) * (i - 1))
    else:
        r = int(rng.integers(1, 420))
        s = np.where(i <= r, 10.0 ** (-rng.uniform(0, 2) * (i - 1) / max(r, 1)), 0.0)
        s[r:] = 10.0 ** -rng.uniform(5, 12) / i[r:]
    if rng.random() < 0.3:
        s = np.maximum(s, 10.0 ** -rng.uniform(5, 12))
    return np.sort(s)[::-1] / s.max(), fam


def _pairs_chunk(count, seed, sizes):
    """One host thread's share of make_pairs: its own handle and stream."""
    rng = np.random.default_rng(seed)
    h = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    st = torch.cuda.Stream()
    X = np.zeros((count, 18), dtype=np.float32)
    y = np.zeros(count, dtype=np.int32)
    fams = np.zeros(count, dtype=np.int32)
    big = torch.zeros(4 * max(sizes) * max(sizes), dtype=torch.float32, device="cuda")
    try:
        with torch.cuda.stream(st):
            for t in range(count):
                n = int(rng.choice(sizes))
                m = int(n * rng.choice([1, 2, 4]))
                A = big[: m * n].view(m, n)
                s, fams[t] = spectrum(rng, n)
                A.zero_()
                A.diagonal().copy_(torch.from_numpy(s.astype(np.float32)).to("cuda", non_blocking=True))
                eps = float(10.0 ** -rng.uniform(1.5, 7))
                sk = int(rng.integers(0, 2 ** 31))
                st.synchronize()                     # the features run on the default stream
                X[t] = rk.re_mlp_features(h, A, eps, sk)
                res, _ = rk.re_rank_estimate(h, A, eps, rk.RE_GAUSSIAN, sk, sigma_cap=0, stream=st)
                y[t] = int(np.log2(res.final_s // 8))
    finally:
        rk.re_destroy(h)
    return X, y, fams


def make_pairs(count, seed, sizes, threads=4):
    """Features of the s = 16 sketch and the plain ladder's width class for
    `count` diagonal matrices (n from `sizes`, m = n, 2n or 4n).  Host threads
    (each with its own handle and stream) overlap the per-call latencies; thread
    j draws from the seed sequence (seed, j), so the pairs do not depend on timing."""
    per = [count // threads + (1 if j < count % threads else 0) for j in range(threads)]
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda j: _pairs_chunk(per[j], [seed, j], sizes), range(threads)))
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
            np.concatenate([p[2] for p in parts]))


def dense_matrix(m, n, s, seed, buf):
    """A = U diag(s) V^T (FP32, on the GPU, in the first m n entries of buf) with
    U, V products of 8 seeded Householder reflectors and random signs, built by
    rank-one updates of the signed diagonal (no m x m or n x n factor is formed)."""
    g = torch.Generator(device="cuda")
    g.manual_seed(int(seed))
    k = min(m, n)
    C = buf[: m * n].view(m, n)
    C.zero_()
    sign = torch.randint(0, 2, (k,), generator=g, device="cuda").to(torch.float32) * 2 - 1
    C[:k, :k].diagonal().copy_(torch.from_numpy(s[:k].astype(np.float32)).to("cuda") * sign)
    for _ in range(8):
        v = torch.randn(n, generator=g, device="cuda")
        v /= torch.linalg.vector_norm(v)
        C.addr_(C @ v, v, alpha=-2.0)        # C <- C (I - 2 v v^T)
    for _ in range(8):
        u = torch.randn(m, generator=g, device="cuda")
        u /= torch.linalg.vector_norm(u)
        C.addr_(u, u @ C, alpha=-2.0)        # C <- (I - 2 u u^T) C
    return C


def _heldout_chunk(count, seed, weights, lo, hi):
    rng = np.random.default_rng(seed)
    hp = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    hl = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3, learned=1))
    rk.re_mlp_load(hl, weights)
    st = torch.cuda.Stream()
    rec = {k: np.zeros(count, dtype=np.int64) for k in ("m", "n", "fam", "cls_true", "plain_passes",
                                                      "learned_passes", "same_rank", "same_width")}
    feats = np.zeros((count, 18), dtype=np.float32)
    ms = np.zeros((count, 2))
    buf = torch.empty(hi * hi, dtype=torch.float32, device="cuda")
    try:
        with torch.cuda.stream(st):
            for t in range(count):
                m, n = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
                s, fam = spectrum(rng, min(m, n))
                A = dense_matrix(m, n, s, rng.integers(0, 2 ** 62), buf)
                eps = float(10.0 ** -rng.uniform(1.5, 6))   # the FP32 matrix resolves to about 1e-7
                sk = int(rng.integers(0, 2 ** 31))
                st.synchronize()
                feats[t] = rk.re_mlp_features(hp, A, eps, sk)
                t1 = time.perf_counter()
                rp, _ = rk.re_rank_estimate(hp, A, eps, rk.RE_GAUSSIAN, sk, sigma_cap=0, stream=st)
                t2 = time.perf_counter()
                rl, _ = rk.re_rank_estimate(hl, A, eps, rk.RE_GAUSSIAN, sk, sigma_cap=0, stream=st)
                t3 = time.perf_counter()
                ms[t] = ((t2 - t1) * 1e3, (t3 - t2) * 1e3)
                rec["m"][t], rec["n"][t], rec["fam"][t] = m, n, fam
                rec["cls_true"][t] = int(np.log2(rp.final_s // 8))
                rec["plain_passes"][t], rec["learned_passes"][t] = rp.passes, rl.passes
                rec["same_rank"][t] = int(rp.rank == rl.rank and rp.flags == rl.flags)
                rec["same_width"][t] = int(rp.final_s == rl.final_s)
    finally:
        rk.re_destroy(hp)
        rk.re_destroy(hl)
    return rec, feats, ms


def heldout_dense(count, seed, weights, lo=1024, hi=16384, threads=3):
    """The held-out evaluation on the dense path: for `count` dense matrices with
    m, n uniform on [lo, hi], the plain ladder and the learned ladder (BF16x3
    tensor-core sketch) are both run and their passes over A, ranks and widths
    recorded; the features are those the learned ladder computes.  Wall times
    per call are host-side and include the other threads' contention."""
    per = [count // threads + (1 if j < count % threads else 0) for j in range(threads)]
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda j: _heldout_chunk(per[j], [seed, j], weights, lo, hi), range(threads)))
    rec = {k: np.concatenate([p[0][k] for p in parts]) for k in parts[0][0]}
    return rec, np.concatenate([p[1] for p in parts]), np.concatenate([p[2] for p in parts])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=200000)
    ap.add_argument("--heldout", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--out", default=os.path.join(HERE, "proposal.remlp"))
    ap.add_argument("--report", default=None)
    a = ap.parse_args()
    build.build()
    h = rk.re_create(0, rk.make_opts(precision=rk.RE_PREC_BF16X3))
    t0 = time.time()
    Xtr, ytr, ftr = make_pairs(a.samples, 1, [1024, 2048, 4096])
    t_data = time.time() - t0
    rk.re_mlp_init(h, 7)
    t1 = time.time()
    losses = rk.re_mlp_train(h, Xtr, ytr, epochs=a.epochs, batch=256, lr=2e-3, weight_decay=1e-5, seed=3)
    t_train = time.time() - t1
    rk.re_mlp_save(h, a.out)
    t2 = time.time()
    rec, Xte, ms = heldout_dense(a.heldout, 2, a.out)
    t_held = time.time() - t2
    ms_p, ms_l = float(ms[:, 0].mean()), float(ms[:, 1].mean())
    cls, _ = rk.re_mlp_predict(h, Xte)
    yte = rec["cls_true"]
    rep = {"train_samples": int(a.samples), "train_sizes": "n in {1024, 2048, 4096}, m = n, 2n or 4n, diagonal",
           "train_family_histogram": dict(zip(FAMILIES, np.bincount(ftr, minlength=len(FAMILIES)).tolist())),
           "label_histogram": np.bincount(ytr, minlength=12).tolist(),
           "data_seconds": t_data, "train_seconds": t_train, "epochs": a.epochs,
           "first_loss": float(losses[0]), "final_loss": float(losses[-1]),
           "heldout": int(a.heldout), "heldout_sizes": "dense U diag(sigma) V^T, m and n uniform on [1024, 16384]",
           "heldout_seconds": t_held,
           "heldout_exact_class": float(np.mean(cls == yte)),
           "heldout_at_or_above": float(np.mean(cls >= yte)),
           "heldout_identical_rank_and_flags": float(np.mean(rec["same_rank"])),
           "heldout_identical_width": float(np.mean(rec["same_width"])),
           "heldout_plain_mean_passes": float(np.mean(rec["plain_passes"])),
           "heldout_learned_mean_passes": float(np.mean(rec["learned_passes"])),
           "heldout_plain_ms_mean": ms_p, "heldout_learned_ms_mean": ms_l,
           "heldout_class_histogram": np.bincount(yte, minlength=12).tolist()}
    print(json.dumps(rep))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    rk.re_destroy(h)


if __name__ == "__main__":
    main()
