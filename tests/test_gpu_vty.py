"""The augmented product fused with C = V^T y (sp_spmv_vty): y and z against
the oracle's product, C against the oracle's inner products of V with the
oracle's y, within the bound the arithmetic allows; y bit-identical to
sp_spmv's (the same row sums and epilogue)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import U53, assert_close, gamma, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    return gen.irregular_band(9001, lmin=0, lmax=48, band=500, seed=23)


@pytest.mark.parametrize("C,sigma", [(32, 256), (64, 1), (7, 1)])
@pytest.mark.parametrize("w,m", [(1, 1), (1, 8), (2, 3), (4, 5), (8, 8), (3, 2)])
def test_vty_matches_oracle(cuda_ok, band, C, sigma, w, m):
    A = band
    rng = np.random.default_rng(w * 10 + m + C)
    X, Y0, Z0 = (rng.uniform(-1, 1, (A.nrows, w)) for _ in range(3))
    V = rng.uniform(-1, 1, (A.nrows, m))
    gam = rng.uniform(-1, 1, w) if w > 1 else 0.25
    mat = sellcs.SellMatrix(A, C=C, sigma=sigma)
    x, y, z, v = (torch.from_numpy(a).cuda() for a in (X, Y0.copy(), Z0.copy(), V))
    if w == 3:  # rows of 3 doubles are not whole 16-byte vectors: refused, nothing written
        Cd = torch.full((m, w), float("nan"), dtype=torch.float64, device="cuda")
        with pytest.raises(sellcs.SpError) as e:
            sellcs.spmv_vty(mat, x, y, v, Cd, alpha=0.5, gamma=gam, beta=-1.5)
        assert e.value.code == sellcs.SP_ERR_UNSUPPORTED
        return
    Cd = torch.full((m, w), float("nan"), dtype=torch.float64, device="cuda")
    sellcs.spmv_vty(mat, x, y, v, Cd, alpha=0.5, gamma=gam, beta=-1.5, z=z, delta=0.9, eta=0.1)
    torch.cuda.synchronize()
    kw = dict(alpha=0.5, gamma=gam, beta=-1.5, y0=Y0)
    yr, _, zr = oracle.spmmv(A, X, **kw, delta=0.9, eta=0.1, z0=Z0)
    sc = oracle.spmmv_scale(A, X, **kw)
    tol = tol_for("f64", "f64", 0)
    yg = y.cpu().numpy()
    assert_close(yg, yr, sc, tol, "vty y")
    assert_close(z.cpu().numpy(), zr, 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + sc), tol, "vty z")
    # C = V^T y: the propagated error of y plus the float64 accumulation
    Cr = oracle.tsmttsm(V, yr)
    e = tol * sc
    bound = np.abs(V).T @ e + (gamma(A.nrows + 2100, U53) + 1e-15) * (np.abs(V).T @ (np.abs(yr) + e))
    assert_close(Cd.cpu().numpy(), Cr, bound, 1.0, "vty C")
    # the same y bits as sp_spmv
    y2, z2 = torch.from_numpy(Y0.copy()).cuda(), torch.from_numpy(Z0.copy()).cuda()
    sellcs.spmv(mat, x, y2, alpha=0.5, gamma=gam, beta=-1.5, z=z2, delta=0.9, eta=0.1)
    torch.cuda.synchronize()
    # the fused form is a variant of the same kernel: same row loops, same epilogue
    assert torch.equal(y2, y) and torch.equal(z2, z)
    mat.close()


def test_vty_arguments(cuda_ok, band):
    A = band
    mat = sellcs.SellMatrix(A, C=32, sigma=1)
    x = torch.rand(A.nrows, 2, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    V = torch.rand(A.nrows, 9, dtype=torch.float64, device="cuda")
    Cd = torch.zeros(9, 2, dtype=torch.float64, device="cuda")
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv_vty(mat, x, y, V, Cd)  # m = 9 > 8
    assert e.value.code == sellcs.SP_ERR_UNSUPPORTED
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv_vty(mat, x, y, y, Cd[:2])  # V is y
    assert e.value.code == sellcs.SP_ERR_ARG
    mat.close()


@pytest.mark.parametrize("m", [1, 4, 8])
def test_vty_full_size(cuda_ok, m):
    """The irregular N = 2^21 workload at SELL-32-256 (the launch configuration
    of the product benchmark) with V of m columns: y and z element by element,
    C within its bound, all against the oracle."""
    A, X, Y0, Z0 = gen.workload_irregular()
    rng = np.random.default_rng(77 + m)
    V = rng.uniform(-0.5, 0.5, (A.nrows, m))
    mat = sellcs.SellMatrix(A, C=32, sigma=256)
    x, y, z, v = (torch.from_numpy(a).cuda() for a in (X, Y0.copy(), Z0.copy(), V))
    Cd = torch.full((m, 1), float("nan"), dtype=torch.float64, device="cuda")
    kw = dict(alpha=0.5, gamma=0.1, beta=1.0)
    sellcs.spmv_vty(mat, x, y, v, Cd, **kw, z=z, delta=0.9, eta=0.1)
    torch.cuda.synchronize()
    yr, _, zr = oracle.spmmv(A, X, **kw, y0=Y0, delta=0.9, eta=0.1, z0=Z0)
    sc = oracle.spmmv_scale(A, X, **kw, y0=Y0)
    tol = tol_for("f64", "f64", 0)
    assert_close(y.cpu().numpy(), yr, sc, tol, "vty y")
    assert_close(z.cpu().numpy(), zr, 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + sc), tol, "vty z")
    y2, e = np.reshape(yr, (A.nrows, 1)), np.reshape(tol * sc, (A.nrows, 1))
    Cr = oracle.tsmttsm(V, y2)
    bound = np.abs(V).T @ e + (gamma(A.nrows + 2100, U53) + 1e-15) * (np.abs(V).T @ (np.abs(y2) + e))
    assert_close(Cd.cpu().numpy(), Cr, bound, 1.0, "vty C")
    mat.close()
