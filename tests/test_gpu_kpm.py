"""KPM moments on the fused product (sp_kpm_moments): the Chebyshev loop with
two moments per product from the fused <y,y> and <x,y>, against the oracle's
moments by definition (one inner product per moment) and against closed forms
(eigenvector starts: mu_k = T_k(lambda~) ||v||^2)."""
import numpy as np
import pytest
import torch
from numpy.polynomial import chebyshev as npcheb

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import to_dev
from workloads import generators as gen

pytestmark = pytest.mark.gpu

A_SCALE = 1.01 * (6 + 8.25)  # Gershgorin bound of the Anderson matrix (disorder 16.5)


@pytest.mark.parametrize("nmom", [1, 2, 3, 4, 5, 64, 101])
@pytest.mark.parametrize("w", [1, 4])
def test_kpm_matches_oracle(cuda_ok, nmom, w):
    A = gen.anderson3d(16, seed=51)
    m = sellcs.SellMatrix(A, C=32, sigma=1)
    X = gen.block_vector(A.nrows, w, 52)
    mu = sellcs.kpm_moments(m, to_dev(X), nmom, A_SCALE, 0.0)
    ref = oracle.kpm_moments(A, X, nmom, A_SCALE, 0.0)
    scale = (X * X).sum(0)
    # Chebyshev recurrences with the spectrum inside [-1, 1] are stable: the
    # error grows at most linearly with k (float64: 1e-13 per step, generous)
    k = np.arange(nmom)[:, None]
    assert np.all(np.abs(mu - ref) <= 1e-13 * (k + 1) ** 2 * scale + 1e-300), np.max(np.abs(mu - ref) / scale)


def test_kpm_shift_and_eigenvector_closed_form(cuda_ok):
    s = 40
    A = gen.laplace2d(s, 0.0)
    th = np.pi / (s + 1)
    a, b = 4.2, 4.0  # spectrum [0, 8] into [-1, 1]
    modes = [(1, 1), (7, 30), (40, 40)]
    V = np.stack([gen.laplace2d_mode(s, p, q) for p, q in modes], axis=1)
    lam = np.array([(4 - 2 * np.cos(p * th) - 2 * np.cos(q * th) - b) / a for p, q in modes])
    m = sellcs.SellMatrix(A, C=16, sigma=64)
    mu = sellcs.kpm_moments(m, to_dev(V), 80, a, b)
    nv = (V * V).sum(0)
    for c in range(3):
        ref = npcheb.chebval(lam[c], np.eye(80)) * nv[c]
        np.testing.assert_allclose(mu[:, c], ref, rtol=0, atol=1e-11 * nv[c])


def test_kpm_float32_vectors(cuda_ok):
    A = gen.anderson3d(16, seed=53)
    m = sellcs.SellMatrix(A, C=32, sigma=1, dtype="f32")
    X = gen.block_vector(A.nrows, 2, 54).astype(np.float32).astype(np.float64)
    mu = sellcs.kpm_moments(m, to_dev(X, torch.float32), 40, A_SCALE, 0.0)
    ref = oracle.kpm_moments(A, X, 40, A_SCALE, 0.0)
    scale = (X * X).sum(0)
    # float32 products and vectors: about 2^-24 per step, growing with k
    k = np.arange(40)[:, None]
    assert np.all(np.abs(mu - ref) <= 2.0 ** -24 * 8 * (k + 1) * scale)


def test_kpm_rejects_bad_arguments(cuda_ok):
    A = gen.laplace2d(8, 0.0)
    m = sellcs.SellMatrix(A, C=8, sigma=1)
    x = to_dev(np.ones((A.nrows, 1)))
    with pytest.raises(sellcs.SpError):
        sellcs.kpm_moments(m, x, 0, 1.0, 0.0)
    with pytest.raises(sellcs.SpError):
        sellcs.kpm_moments(m, x, 4, 0.0, 0.0)
    R = gen.CSR(4, 6, np.array([0, 1, 2, 3, 4]), np.array([0, 1, 2, 3], np.int32), np.ones(4))
    mr = sellcs.SellMatrix(R, C=4, sigma=1)
    with pytest.raises(sellcs.SpError):
        sellcs.kpm_moments(mr, to_dev(np.ones((4, 1))), 4, 1.0, 0.0)
