"""Permuted space (SP_MAT_PERMUTED_SPACE): vectors in SELL row order, column
indices stored as slots.  Moving x, y0, z0 into SELL order (sp_mat_permute),
multiplying, and moving y, z back gives y, z and the dots of the oracle's
augmented product on the user's vectors (within the tolerances of the other
parity tests), and the same bits as the product in the user's order (same
entries, same order in every row, same slot order of the dot accumulation);
the CSR export returns the user's matrix."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import assert_close, dot_bound, to_dev, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def matrix():
    return gen.irregular_band(20_001, lmin=0, lmax=30, band=300, seed=61)


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 64), (8, 20_001)])
@pytest.mark.parametrize("w", [1, 3, 16])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_permuted_space_matches_user_order(cuda_ok, matrix, C, sigma, w, xdt):
    A = matrix
    tdt = torch.float64 if xdt == "f64" else torch.float32
    vdt = xdt
    mu = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=vdt)
    mp = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=vdt, permuted=True)
    rng = np.random.default_rng(62)
    Xh, Y0h, Z0h = (rng.uniform(-1, 1, (A.nrows, w)) for _ in range(3))
    if xdt == "f32":
        Xh, Y0h, Z0h = (v.astype(np.float32).astype(np.float64) for v in (Xh, Y0h, Z0h))
    X, Y0, Z0 = (to_dev(v, tdt) for v in (Xh, Y0h, Z0h))
    kw = dict(alpha=0.5, gamma=0.25, beta=-1.5, dot_yy=True, dot_xy=True, dot_xx=True, delta=0.9, eta=0.1)
    y, z = Y0.clone(), Z0.clone()
    d = sellcs.spmv(mu, X, y, z=z, **kw)
    xp, yp, zp = (torch.empty_like(v) for v in (X, Y0, Z0))
    for src, dst in ((X, xp), (Y0, yp), (Z0, zp)):
        sellcs.mat_permute(mp, dst, src, True)
    dp = sellcs.spmv(mp, xp, yp, z=zp, **kw)
    yb, zb = torch.empty_like(y), torch.empty_like(z)
    sellcs.mat_permute(mp, yb, yp, False)
    sellcs.mat_permute(mp, zb, zp, False)
    torch.cuda.synchronize()
    # against the oracle, in the user's order
    vals = oracle.round_values(A.val, vdt)
    okw = dict(val=vals, alpha=0.5, gamma=0.25, beta=-1.5, y0=Y0h)
    yr, dr, zr = oracle.spmmv(A, Xh, **okw, dot_yy=True, dot_xy=True, dot_xx=True, delta=0.9, eta=0.1, z0=Z0h)
    sc = oracle.spmmv_scale(A, Xh, **okw)
    tol = tol_for(vdt, xdt, int(np.diff(A.rowptr).max()))
    if xdt == "f32":
        sc = sc + np.abs(yr)
    yg = yb.double().cpu().numpy().reshape(A.nrows, w)
    assert_close(yg, yr, sc, tol, "permuted-space y vs oracle")
    zsc = 0.9 * np.abs(Z0h) + 0.1 * (np.abs(yr) + sc)
    assert_close(zb.double().cpu().numpy().reshape(A.nrows, w), zr, zsc, tol + (2 ** -24 if xdt == "f32" else 0),
                 "permuted-space z vs oracle")
    dpn = dp.cpu().numpy()
    for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
        assert_close(dpn[q * w:(q + 1) * w], dr[q * w:(q + 1) * w], dot_bound(name, yr, Xh, tol * sc, xdt, A.nrows),
                     1.0, f"permuted-space {name} vs oracle")
    # and the same bits as the user-order product
    assert torch.equal(yb, y) and torch.equal(zb, z)
    assert torch.equal(dp, d)


def test_permuted_space_round_trips(cuda_ok, matrix):
    A = matrix
    mp = sellcs.SellMatrix(A, C=16, sigma=256, permuted=True)
    rp = np.zeros(A.nrows + 1, np.int64)
    col = np.zeros(A.nnz, np.int32)
    val = np.zeros(A.nnz)
    sellcs.check(sellcs.lib().sp_mat_to_csr(mp.handle, rp.ctypes.data, col.ctypes.data, val.ctypes.data, None),
                 "sp_mat_to_csr")
    assert np.array_equal(rp, A.rowptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)
    x = to_dev(np.random.default_rng(63).uniform(-1, 1, (A.nrows, 5)))
    xp, xb = torch.empty_like(x), torch.empty_like(x)
    sellcs.mat_permute(mp, xp, x, True)
    sellcs.mat_permute(mp, xb, xp, False)
    torch.cuda.synchronize()
    assert torch.equal(xb, x)
    assert not torch.equal(xp, x)  # sigma = 256 really permutes
    with pytest.raises(sellcs.SpError):
        sellcs.mat_permute(mp, x, x, True)  # in place is refused


def test_permuted_space_rejects_adjoint(cuda_ok, matrix):
    mp = sellcs.SellMatrix(matrix, C=32, sigma=1, permuted=True)
    g = to_dev(np.ones((matrix.nrows, 1)))
    with pytest.raises(sellcs.SpError):
        sellcs.spmv_adjoint(mp, g, x=g, dvals=torch.empty(matrix.nnz, dtype=torch.float64, device="cuda"))
