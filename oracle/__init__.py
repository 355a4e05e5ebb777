"""FP64 CPU oracle for randomized numerical-rank estimation (Meier & Nakatsukasa,
"Fast Randomized Numerical Rank Estimation for Numerically Low-Rank Matrices").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the CUDA library and its Python binding) never
imports, links or executes anything here, and this package imports nothing from
the product package.

Contents
--------
``rng``        counter-based generator (Philox4x32-10, Box-Muller normals rounded
               to BF16, random signs, keyed Feistel sampling, the HRTT's
               CountSketch hashing built on them) written from the
               published definitions; the CUDA side has its own implementation of
               the same specification, so both draw identical X and Y.
``algorithm1`` Algorithm 1 (Sec. 5) step by step in FP64 with numpy: the sketch
               matrices written out densely, A·X and Θ·(A·X) by matrix products,
               singular values by LAPACK, read-off by Definition 1.
``algorithm3`` Algorithm 3 (Sec. 5.1): rank estimation combined with the
               randomized rangefinder -- the Frobenius criterion on the
               sketched singular values picks r, then a Householder thin QR of
               the first r + p columns of A X and B = Q^T A.
``mlp``        the sketch-size proposal network's forward/backward in FP64
               (plain numpy), used to check the GPU gradients.

Parity status: every function here is pinned by ``-m "not gpu"`` tests against
published known-answer vectors, closed forms, library routines or the paper's
bounds; none is "parity unpinned".
"""
