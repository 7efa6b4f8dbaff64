"""Pins of the oracle's KPM moments mu_k = <x, T_k(A~) x>, A~ = (A - b I)/a,
against things other than its own recurrence:

* the spectral form sum_i (v_i . x)^2 T_k(lambda_i) over the eigenpairs of the
  dense A~ (numpy eigh), with T_k evaluated by numpy's Chebyshev series;
* an eigenvector start: mu_k = T_k(lambda~) ||v||^2 (2D Laplacian sine mode).
"""
import numpy as np
from numpy.polynomial import chebyshev as npcheb

import oracle
from tests.test_oracle_format import random_csr
from tests.test_oracle_spmmv import dense
from workloads import generators as gen


def _symmetric_csr(n, density, rng):
    A = random_csr(n, n, density, rng)
    D = dense(A)
    S = D + D.T + np.diag(rng.uniform(-2, 2, n))
    rows, cols = np.nonzero(S)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return gen.CSR(n, n, rowptr, cols.astype(np.int32), S[rows, cols])


def test_moments_match_spectral_form():
    rng = np.random.default_rng(7)
    for n, w in ((12, 1), (30, 3), (45, 2)):
        A = _symmetric_csr(n, 0.15, rng)
        D = dense(A)
        a, b = 1.1 * np.abs(np.linalg.eigvalsh(D)).max() + 0.5, 0.3
        X = rng.uniform(-1, 1, (n, w))
        mu = oracle.kpm_moments(A, X, 24, a, b)
        lam, V = np.linalg.eigh((D - b * np.eye(n)) / a)
        for c in range(w):
            wts = (V.T @ X[:, c]) ** 2
            for k in range(24):
                ek = np.zeros(k + 1)
                ek[k] = 1.0
                ref = float(wts @ npcheb.chebval(lam, ek))
                assert abs(mu[k, c] - ref) <= 1e-11 * (wts.sum() + 1.0), (n, c, k, mu[k, c], ref)


def test_eigenvector_start_gives_chebyshev_of_eigenvalue():
    s = 20
    A = gen.laplace2d(s, 0.0)
    th = np.pi / (s + 1)
    a, b = 4.2, 4.0  # spectrum [0, 8] into [-1, 1]
    for p, q in ((1, 1), (4, 9), (20, 20)):
        v = gen.laplace2d_mode(s, p, q)
        lam = (4.0 - 2 * np.cos(p * th) - 2 * np.cos(q * th) - b) / a
        mu = oracle.kpm_moments(A, v, 40, a, b)[:, 0]
        ref = npcheb.chebval(lam, np.eye(40)) * float(v @ v)
        np.testing.assert_allclose(mu, ref, rtol=0, atol=1e-11 * float(v @ v))
