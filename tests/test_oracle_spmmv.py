"""Pins of the oracle's augmented SpMMV (CPU only).

* Dense brute force: numpy's dense matmul on the densified matrix for every
  subset of the augmentation flags, on non-symmetric rectangular-free random
  matrices (a transposed operand, a dropped term or a wrong sign fails here).
* Closed forms: sine modes of the 3D Dirichlet Laplacian and plane waves of the
  clean periodic lattice are eigenvectors, so y, <x,x>, <x,y>, <y,y> are known
  without any code; the golden 5x5 product is worked by hand.
* y is not read when the beta flag is off.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.test_oracle_format import random_csr
from workloads import generators as gen


def dense(A):
    D = np.zeros((A.nrows, A.ncols))
    for i in range(A.nrows):
        seg = slice(A.rowptr[i], A.rowptr[i + 1])
        D[i, A.col[seg]] = A.val[seg]
    return D


FLAGS = ["scale", "shift", "vshift", "axpby", "dot_yy", "dot_xy", "dot_xx", "chain"]


def _flag_sets():
    for bits in range(1 << len(FLAGS)):
        f = {n for k, n in enumerate(FLAGS) if bits >> k & 1}
        if "shift" in f and "vshift" in f:
            continue
        yield f


def _run(A, X, Y0, Z0, f, alpha=0.7, beta=-1.3, gs=0.25, gv=None, delta=0.9, eta=0.1):
    w = X.shape[1]
    gv = np.linspace(-0.5, 0.5, w) if gv is None else gv
    gamma = gs if "shift" in f else (gv if "vshift" in f else None)
    return oracle.spmmv(A, X, alpha=alpha if "scale" in f else None, gamma=gamma,
                        beta=beta if "axpby" in f else None, y0=Y0 if "axpby" in f else None,
                        dot_yy="dot_yy" in f, dot_xy="dot_xy" in f, dot_xx="dot_xx" in f,
                        delta=delta if "chain" in f else None, eta=eta if "chain" in f else None,
                        z0=Z0 if "chain" in f else None)


@pytest.mark.parametrize("N,w", [(7, 1), (13, 3), (33, 4)])
def test_dense_bruteforce_all_flags(N, w):
    rng = np.random.default_rng(N * 10 + w)
    A = random_csr(N, N, 0.3, rng)
    D = dense(A)
    X = rng.uniform(-1, 1, (N, w))
    Y0 = rng.uniform(-1, 1, (N, w))
    Z0 = rng.uniform(-1, 1, (N, w))
    gv = rng.uniform(-1, 1, w)
    n = 0
    for f in _flag_sets():
        alpha = 0.7 if "scale" in f else 1.0
        beta = -1.3 if "axpby" in f else 0.0
        gam = np.full(w, 0.25) if "shift" in f else (gv if "vshift" in f else np.zeros(w))
        ref = alpha * (D @ X - X * gam[None, :]) + beta * (Y0 if "axpby" in f else 0.0)
        y, dot, z = _run(A, X, Y0, Z0, f, gv=gv)
        tol = 1e-15 * (np.abs(D) @ np.abs(X) + np.abs(X) + np.abs(Y0) + 1)
        assert np.all(np.abs(y - ref) <= tol), f
        exp = {"dot_yy": (ref * ref).sum(0), "dot_xy": (X * ref).sum(0), "dot_xx": (X * X).sum(0)}
        for s, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
            got = dot[s * w:(s + 1) * w]
            if name in f:
                np.testing.assert_allclose(got, exp[name], rtol=1e-14, atol=1e-14)
            else:
                assert np.all(np.isnan(got))  # untouched
        if "chain" in f:
            np.testing.assert_allclose(z, 0.9 * Z0 + 0.1 * ref, rtol=1e-15, atol=1e-15)
        else:
            assert z is None
        n += 1
    assert n == 192


def test_rectangular_plain():
    rng = np.random.default_rng(1)
    A = random_csr(9, 17, 0.4, rng)
    A.ncols = 17
    X = rng.uniform(-1, 1, (17, 2))
    y, _, _ = oracle.spmmv(A, X)
    np.testing.assert_allclose(y, dense(A) @ X, rtol=1e-15, atol=1e-15)


def test_beta_off_does_not_read_y():
    A = gen.laplace3d(4)
    x = np.ones((A.nrows, 1))
    y0 = np.full((A.nrows, 1), np.nan)
    y, _, _ = oracle.spmmv(A, x, y0=y0)  # beta None -> y0 ignored
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("p,q,r", [(1, 1, 1), (3, 7, 2), (32, 1, 16)])
def test_laplace3d_sine_modes(p, q, r):
    n = 32
    A = gen.laplace3d(n)
    v = gen.laplace3d_mode(n, p, q, r)
    th = np.pi / (n + 1)
    lam = 6 - 2 * np.cos(p * th) - 2 * np.cos(q * th) - 2 * np.cos(r * th)
    alpha, gamma = 0.5, 0.3
    y, dot, _ = oracle.spmmv(A, v, alpha=alpha, gamma=gamma, dot_yy=True, dot_xy=True, dot_xx=True)
    np.testing.assert_allclose(y[:, 0], alpha * (lam - gamma) * v, rtol=0, atol=1e-13)
    nv = (33 / 2) ** 3
    assert nv == 4492.125
    np.testing.assert_allclose(dot[2], nv, rtol=1e-13)
    np.testing.assert_allclose(dot[1], alpha * (lam - gamma) * nv, rtol=1e-12)
    np.testing.assert_allclose(dot[0], (alpha * (lam - gamma)) ** 2 * nv, rtol=1e-12)


@pytest.mark.parametrize("p,q,r", [(0, 0, 0), (1, 2, 3), (5, 0, 7)])
def test_periodic_lattice_plane_waves(p, q, r):
    n = 16
    A = gen.anderson3d(n, disorder=False)
    v = gen.lattice_plane_wave(n, p, q, r)
    t = 2 * np.pi / n
    lam = -2 * (np.cos(p * t) + np.cos(q * t) + np.cos(r * t))
    y, _, _ = oracle.spmmv(A, v)
    np.testing.assert_allclose(y[:, 0], lam * v, rtol=0, atol=1e-13)


def test_chebyshev_recurrence_on_eigenvector():
    """w_{k+1} = 2 A~ w_k - w_{k-1} with A~ = A/a maps an eigenvector v to
    T_k(lambda/a) v (the scalar Chebyshev recurrence)."""
    n = 12
    A = gen.anderson3d(n, disorder=False)
    v = gen.lattice_plane_wave(n, 1, 2, 0)
    lam = -2 * (np.cos(2 * np.pi / n) + np.cos(4 * np.pi / n) + 1.0)
    a = 1.01 * 6
    w_prev, w_cur = v.copy(), oracle.spmmv(A, v, alpha=1 / a)[0][:, 0]
    for k in range(2, 30):
        w_next = oracle.spmmv(A, w_cur, alpha=2 / a, beta=-1.0, y0=w_prev)[0][:, 0]
        w_prev, w_cur = w_cur, w_next
        Tk = np.cos(k * np.arccos(lam / a))
        np.testing.assert_allclose(w_cur, Tk * v, rtol=0, atol=1e-12)


def test_scale_is_magnitude_bound():
    rng = np.random.default_rng(3)
    A = random_csr(20, 20, 0.3, rng)
    X = rng.uniform(-1, 1, (20, 2))
    Y0 = rng.uniform(-1, 1, (20, 2))
    s = oracle.spmmv_scale(A, X, alpha=2.0, gamma=[0.5, -1.0], beta=3.0, y0=Y0)
    D = dense(A)
    ref = 2.0 * (np.abs(D) @ np.abs(X)) + np.abs(2.0 * np.array([0.5, -1.0]))[None] * np.abs(X) + 3.0 * np.abs(Y0)
    np.testing.assert_allclose(s, ref, rtol=1e-14)


def test_round_values_bf16_and_f32():
    import torch
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.normal(size=10000), rng.uniform(-1e-3, 1e-3, 1000),
                        [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -0.0, 65504.0, 3e38]])
    ref16 = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_values(v, "bf16"), ref16)
    np.testing.assert_array_equal(oracle.round_values(v, "f32"), v.astype(np.float32).astype(np.float64))
    # ties to even at 1.0: spacing 2**-7
    r = oracle.round_values(np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8]), "bf16")
    assert r[0] == 1.0 and r[1] == 1 + 2 ** -6


def test_openmp_timing_variant_matches_single_thread():
    """The all-cores timing baseline (orc_spmmv_omp) computes every row as
    orc_spmmv does: the same y and z bits; the dots differ only by the order
    in which the threads' compensated sums are added."""
    from workloads import generators as gen
    A = gen.irregular_band(3001, lmin=0, lmax=40, band=200, seed=3)
    rng = np.random.default_rng(0)
    X, Y0, Z0 = (rng.uniform(-1, 1, (A.nrows, 2)) for _ in range(3))
    kw = dict(alpha=0.5, gamma=[0.1, -0.2], beta=1.0, y0=Y0, dot_yy=True, dot_xy=True, dot_xx=True, delta=0.9,
              eta=0.1, z0=Z0)
    yr, dr, zr = oracle.spmmv(A, X, **kw)
    for nt in (1, 3, 8):
        got = oracle.spmmv_omp(A, X, nthreads=nt, **kw)
        if got is None:
            pytest.skip("gcc without OpenMP")
        y, d, z = got
        np.testing.assert_array_equal(y, yr)
        np.testing.assert_array_equal(z, zr)
        np.testing.assert_allclose(d, dr, rtol=1e-15, atol=0)
