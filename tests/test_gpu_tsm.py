"""Tall and skinny kernels (sp_tsmttsm, sp_tsmm) against the oracle: the
float64 result within the recursive-summation bound, the Kahan variant close
to the exact sum on cancelling data, bit-identical repeats, the in-place
tsmm, and edge shapes (one row, a partial tile, widths 1 and 32)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (31, 3, 2), (1000, 4, 8), (100_003, 16, 16), (70_001, 32, 5),
                                   (33_333, 1, 32)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tsmttsm(cuda_ok, n, m, k, dt):
    rng = np.random.default_rng(n + m + k)
    tdt = torch.float64 if dt == "f64" else torch.float32
    V, W, X0 = rng.uniform(-1, 1, (n, m)), rng.uniform(-1, 1, (n, k)), rng.uniform(-1, 1, (m, k))
    if dt == "f32":
        V, W, X0 = (a.astype(np.float32).astype(np.float64) for a in (V, W, X0))
    ref = oracle.tsmttsm(V, W, X0, alpha=0.5, beta=-2.0)
    bound = 0.5 * (np.abs(V).T @ np.abs(W)) + 2.0 * np.abs(X0)
    u = U64 if dt == "f64" else 2.0 ** -24
    for kahan in (False, True):
        X = to_dev(X0, tdt)
        sellcs.tsmttsm(X, to_dev(V, tdt), to_dev(W, tdt), 0.5, -2.0, kahan)
        torch.cuda.synchronize()
        got = X.double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1.1 * (n + 4) * u * bound + 1e-300)
        X2 = to_dev(X0, tdt)
        sellcs.tsmttsm(X2, to_dev(V, tdt), to_dev(W, tdt), 0.5, -2.0, kahan)
        assert torch.equal(X, X2)


def test_tsmttsm_kahan_on_cancelling_sums(cuda_ok):
    """Large and small terms of both signs: the compensated sums stay within a
    few units of the exact result where plain sums lose digits."""
    rng = np.random.default_rng(73)
    n = 1 << 20
    V = rng.uniform(-1, 1, (n, 2)) * np.where(rng.uniform(size=(n, 1)) < 0.01, 1e8, 1.0)
    W = np.ones((n, 1))
    exact = np.array([math.fsum(V[:, 0]), math.fsum(V[:, 1])])
    out = {}
    for kahan in (False, True):
        X = torch.zeros(2, 1, dtype=torch.float64, device="cuda")
        sellcs.tsmttsm(X, to_dev(V), to_dev(W), 1.0, 0.0, kahan)
        torch.cuda.synchronize()
        out[kahan] = np.abs(X.cpu().numpy()[:, 0] - exact)
    scale = np.abs(V).sum(0)
    assert np.all(out[True] <= 8 * U64 * scale)
    assert np.all(out[True] <= out[False] + 8 * U64 * scale)


@pytest.mark.parametrize("n,m,k", [(1, 1, 1), (33, 2, 2), (50_001, 8, 8), (50_001, 16, 4), (20_000, 32, 32)])
@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_tsmm(cuda_ok, n, m, k, dt):
    rng = np.random.default_rng(n * 7 + m + k)
    tdt = torch.float64 if dt == "f64" else torch.float32
    V, X, W0 = rng.uniform(-1, 1, (n, m)), rng.uniform(-1, 1, (m, k)), rng.uniform(-1, 1, (n, k))
    if dt == "f32":
        V, X, W0 = (a.astype(np.float32).astype(np.float64) for a in (V, X, W0))
    u = U64 if dt == "f64" else 2.0 ** -24
    ref = oracle.tsmm(V, X, W0, alpha=1.5, beta=0.25)
    bound = 1.5 * (np.abs(V) @ np.abs(X)) + 0.25 * np.abs(W0)
    W = to_dev(W0, tdt)
    sellcs.tsmm(W, to_dev(V, tdt), to_dev(X, tdt), 1.5, 0.25)
    torch.cuda.synchronize()
    assert np.all(np.abs(W.double().cpu().numpy() - ref) <= 1.1 * (m + 3) * u * bound + 1e-300)
    if m == k:
        # in place: V <- 1.5 V X + 0.25 V
        Vd = to_dev(V, tdt)
        sellcs.tsmm(Vd, Vd, to_dev(X, tdt), 1.5, 0.25)
        torch.cuda.synchronize()
        ref2 = oracle.tsmm(V, X, V, alpha=1.5, beta=0.25)
        bound2 = 1.5 * (np.abs(V) @ np.abs(X)) + 0.25 * np.abs(V)
        assert np.all(np.abs(Vd.double().cpu().numpy() - ref2) <= 1.1 * (m + 3) * u * bound2 + 1e-300)


def test_tsm_argument_errors(cuda_ok):
    V = torch.zeros(10, 33, dtype=torch.float64, device="cuda")
    W = torch.zeros(10, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(sellcs.SpError):
        sellcs.tsmttsm(torch.zeros(33, 4, dtype=torch.float64, device="cuda"), V, W)  # m > 32
    with pytest.raises(sellcs.SpError):
        sellcs.tsmttsm(torch.zeros(3, 4, dtype=torch.float64, device="cuda"), W, W)  # X shape
    Vs = torch.zeros(10, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(sellcs.SpError) as e:
        # W a narrower view of V at the same address: not the in-place form (m != k)
        sellcs.tsmm(Vs[:, :3], Vs, torch.zeros(4, 3, dtype=torch.float64, device="cuda"))
    assert e.value.code == sellcs.SP_ERR_ARG
    Vb = torch.zeros(12, 4, dtype=torch.float64, device="cuda")
    with pytest.raises(sellcs.SpError) as e:
        # same leading dimension, rows shifted by two: a partial overlap
        sellcs.tsmm(Vb[2:], Vb[:10], torch.zeros(4, 4, dtype=torch.float64, device="cuda"))
    assert e.value.code == sellcs.SP_ERR_ARG
