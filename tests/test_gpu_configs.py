"""The paper-shaped workloads at full size on the GPU, launched the way
bench.py launches them, against the oracle (every entry) and closed forms.

* 3D 7-point Dirichlet Laplacian 32^3, SELL-32-1, plain y = A x; sine modes.
* Irregular band matrix N = 2^21, SELL-32-256, augmented product with
  <x,y>, <y,y> and the chain (the benchmark workload).
* Anderson lattice 128^3, width-16 row-major block, Chebyshev steps in float64,
  float32 and bfloat16 values; plane waves of the clean lattice.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import U32, assert_close, dot_bound, run_case, to_dev
from workloads import generators as gen

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_laplace_32_full(cuda_ok):
    A, X = gen.workload_laplace()
    run_case(A, 32, 1, 1, set())
    m = sellcs.SellMatrix(A, C=32, sigma=1)
    for p, q, r in [(1, 1, 1), (5, 9, 2), (32, 32, 32)]:
        v = gen.laplace3d_mode(32, p, q, r)
        th = np.pi / 33
        lam = 6 - 2 * np.cos(p * th) - 2 * np.cos(q * th) - 2 * np.cos(r * th)
        y = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
        dot = sellcs.spmv(m, to_dev(v), y, alpha=0.5, gamma=0.3, dot_yy=True, dot_xy=True, dot_xx=True)
        torch.cuda.synchronize()
        np.testing.assert_allclose(y.cpu().numpy(), 0.5 * (lam - 0.3) * v, rtol=0, atol=1e-13)
        nv = (33 / 2) ** 3
        d = dot.cpu().numpy()
        np.testing.assert_allclose(d, [(0.5 * (lam - 0.3)) ** 2 * nv, 0.5 * (lam - 0.3) * nv, nv], rtol=1e-12)


def test_irregular_full_augmented(cuda_ok):
    A, X, Y0, Z0 = gen.workload_irregular()
    m = sellcs.SellMatrix(A, C=32, sigma=256)
    x, y, z = to_dev(X), to_dev(Y0), to_dev(Z0)
    dot = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    sellcs.spmv(m, x, y, alpha=0.5, gamma=0.1, beta=1.0, dot_xy=True, dot_yy=True, z=z, delta=0.9, eta=0.1,
                dot=dot)
    torch.cuda.synchronize()
    yr, dr, zr = oracle.spmmv(A, X, alpha=0.5, gamma=0.1, beta=1.0, y0=Y0, dot_xy=True, dot_yy=True, delta=0.9,
                              eta=0.1, z0=Z0)
    s = oracle.spmmv_scale(A, X, alpha=0.5, gamma=0.1, beta=1.0, y0=Y0)
    yg = y.cpu().numpy()
    assert_close(yg, yr, s, 1e-12, "y")
    assert_close(z.cpu().numpy(), zr, 0.9 * np.abs(Z0) + 0.1 * s, 1e-12, "z")
    d = dot.cpu().numpy()
    assert np.isnan(d[2])
    e = 1e-12 * s
    assert abs(d[0] - dr[0]) <= dot_bound("dot_yy", yr, X, e, "f64", A.nrows)[0]
    assert abs(d[1] - dr[1]) <= dot_bound("dot_xy", yr, X, e, "f64", A.nrows)[0]
    # consistency pin: dots recomputed on the host from the returned y
    assert abs(d[0] - float((yg * yg).sum())) <= 1e-13 * float((yg * yg).sum())
    assert abs(d[1] - float((X * yg).sum())) <= 1e-13 * float(np.abs(X * yg).sum())


@pytest.fixture(scope="module")
def anderson():
    return gen.workload_anderson()


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f64"), ("bf16", "f64"), ("f32", "f32"),
                                     ("bf16", "f32")])
def test_anderson_chebyshev_steps(cuda_ok, anderson, vdt, xdt):
    """Two Chebyshev steps w1 = A~ w0, w2 = 2 A~ w1 - w0 (A~ = A / a), width 16,
    each compared with the oracle applied to the GPU's own previous iterate."""
    A, X = anderson
    a = 1.01 * (6 + 8.25)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    if xdt == "f32":
        X = X.astype(np.float32).astype(np.float64)
    vals = oracle.round_values(A.val, vdt)
    m = sellcs.SellMatrix(A, C=32, sigma=1, dtype=vdt)
    w0 = to_dev(X, tdt)
    w1 = torch.zeros_like(w0)
    sellcs.spmv(m, w0, w1, alpha=1 / a)
    w0h = X
    w1h = w1.double().cpu().numpy()
    ref1 = oracle.spmmv(A, w0h, val=vals, alpha=1 / a)[0]
    s1 = oracle.spmmv_scale(A, w0h, val=vals, alpha=1 / a) + (np.abs(ref1) if xdt == "f32" else 0)
    tol = 1e-12 if vdt == xdt == "f64" else 1.1 * 13 * U32
    assert_close(w1h, ref1, s1, tol, f"T1 {vdt}/{xdt}")
    # w2 = 2/a A w1 - w0 : y holds w0 on entry (beta = -1)
    w2 = w0.clone()
    sellcs.spmv(m, w1, w2, alpha=2 / a, beta=-1.0)
    ref2 = oracle.spmmv(A, w1h, val=vals, alpha=2 / a, beta=-1.0, y0=w0h)[0]
    s2 = oracle.spmmv_scale(A, w1h, val=vals, alpha=2 / a, beta=-1.0, y0=w0h) + (np.abs(ref2) if xdt == "f32" else 0)
    assert_close(w2.double().cpu().numpy(), ref2, s2, tol, f"T2 {vdt}/{xdt}")
    # storage error of the reduced precision against the float64 matrix, stated
    if vdt != "f64":
        exact = oracle.spmmv(A, w0h, alpha=1 / a)[0]
        rel = np.abs(w1h - exact).max() / np.abs(exact).max()
        assert rel < (2 ** -8 if vdt == "bf16" else 2 ** -20)


@pytest.mark.parametrize("vdt", ["f32", "bf16"])
def test_anderson_float32_dots_full(cuda_ok, anderson, vdt):
    """The Anderson workload at full size (N = 2^21, width 16) with float32
    vectors: one step y = A~ x with <y,y>, <x,y>, <x,x>.  Every entry of y and
    every column's three dots against the oracle; the dots within dot_bound,
    whose float part is gamma over SP_DOT_RUN_F32 + 5 additions (the kernel's
    longest float run per lane plus the float lane tree), not over N."""
    A, X = anderson
    a = 1.01 * (6 + 8.25)
    X = X.astype(np.float32).astype(np.float64)
    vals = oracle.round_values(A.val, vdt)
    m = sellcs.SellMatrix(A, C=32, sigma=1, dtype=vdt)
    x = to_dev(X, torch.float32)
    y = torch.zeros_like(x)
    dot = sellcs.spmv(m, x, y, alpha=1 / a, dot_yy=True, dot_xy=True, dot_xx=True)
    torch.cuda.synchronize()
    yr, dr, _ = oracle.spmmv(A, X, val=vals, alpha=1 / a, dot_yy=True, dot_xy=True, dot_xx=True)
    s = oracle.spmmv_scale(A, X, val=vals, alpha=1 / a) + np.abs(yr)
    tol = 1.1 * 13 * U32
    assert_close(y.double().cpu().numpy(), yr, s, tol, f"y {vdt}/f32")
    d = dot.cpu().numpy()
    w = X.shape[1]
    for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
        bound = dot_bound(name, yr, X, tol * s, "f32", A.nrows)
        assert_close(d[q * w:(q + 1) * w], dr[q * w:(q + 1) * w], bound, 1.0, f"{name} {vdt}/f32")
        # the bound is far from vacuous: under 1e-5 of the sum of the terms' magnitudes
        xa = np.abs(X)
        mag = {"dot_yy": yr * yr, "dot_xy": xa * np.abs(yr), "dot_xx": xa * xa}[name].sum(0)
        assert np.all(bound < 1e-5 * mag), (name, float((bound / mag).max()))


def test_clean_lattice_plane_waves_chebyshev(cuda_ok):
    """With the disorder off the plane waves are eigenvectors, so k Chebyshev
    steps give T_k(lambda/a) v exactly (no oracle involved)."""
    n = 128
    A = gen.anderson3d(n, disorder=False)
    a = 1.01 * 6
    modes = [(1, 0, 0), (2, 3, 5), (64, 64, 64), (7, 1, 30)]
    V = np.stack([gen.lattice_plane_wave(n, *pqr) for pqr in modes], axis=1)
    t = 2 * np.pi / n
    lam = np.array([-2 * (np.cos(p * t) + np.cos(q * t) + np.cos(r * t)) for p, q, r in modes])
    m = sellcs.SellMatrix(A, C=32, sigma=1)
    wp = to_dev(V)
    wc = torch.zeros_like(wp)
    sellcs.spmv(m, wp, wc, alpha=1 / a)
    for k in range(2, 12):
        wp2 = wp
        sellcs.spmv(m, wc, wp2, alpha=2 / a, beta=-1.0)  # wp <- 2 A~ wc - wp
        wp, wc = wc, wp2
    torch.cuda.synchronize()
    Tk = np.cos(11 * np.arccos(lam / a))
    np.testing.assert_allclose(wc.cpu().numpy(), V * Tk[None, :], rtol=0, atol=1e-12)
