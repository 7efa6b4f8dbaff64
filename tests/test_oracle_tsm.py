"""Pins of the oracle's tall and skinny kernels: explicit loops with exact
(math.fsum) sums on small blocks, and the transpose identity."""
import math

import numpy as np

import oracle


def test_tsmttsm_against_exact_loops():
    rng = np.random.default_rng(71)
    for n, m, k in ((7, 3, 2), (40, 5, 8), (1, 1, 1)):
        V, W, X0 = rng.uniform(-1, 1, (n, m)), rng.uniform(-1, 1, (n, k)), rng.uniform(-1, 1, (m, k))
        got = oracle.tsmttsm(V, W, X0, alpha=0.75, beta=-1.25)
        for a in range(m):
            for b in range(k):
                ref = 0.75 * math.fsum(V[i, a] * W[i, b] for i in range(n)) - 1.25 * X0[a, b]
                assert abs(got[a, b] - ref) <= 1e-14 * (1 + abs(ref))
    # (V^T W)^T = W^T V
    V, W = rng.uniform(-1, 1, (33, 4)), rng.uniform(-1, 1, (33, 6))
    np.testing.assert_allclose(oracle.tsmttsm(V, W).T, oracle.tsmttsm(W, V), rtol=0, atol=1e-14)


def test_tsmm_against_exact_loops():
    rng = np.random.default_rng(72)
    n, m, k = 9, 4, 3
    V, X, W0 = rng.uniform(-1, 1, (n, m)), rng.uniform(-1, 1, (m, k)), rng.uniform(-1, 1, (n, k))
    got = oracle.tsmm(V, X, W0, alpha=2.0, beta=0.5)
    for i in range(n):
        for b in range(k):
            ref = 2.0 * math.fsum(V[i, a] * X[a, b] for a in range(m)) + 0.5 * W0[i, b]
            assert abs(got[i, b] - ref) <= 1e-14 * (1 + abs(ref))
