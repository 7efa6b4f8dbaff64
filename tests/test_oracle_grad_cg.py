"""Pins of the oracle's derivatives of y = A x and of its CG solvers (CPU only).

* A^T g and the sampled product against dense numpy (transpose and einsum);
* both against float64 central finite differences (h = 1e-6) of the oracle's
  own forward product, on a slice of a power-law matrix;
* CG against the closed-form solution for an eigenvector right-hand side and
  against scipy's sparse direct solver.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle_format import random_csr
from tests.test_oracle_spmmv import dense
from workloads import generators as gen


def test_transpose_and_sampled_dense():
    rng = np.random.default_rng(2)
    A = random_csr(31, 31, 0.2, rng)
    D = dense(A)
    g = rng.normal(size=(31, 3))
    x = rng.normal(size=(31, 3))
    np.testing.assert_allclose(oracle.spmmv_transpose(A, g), D.T @ g, rtol=1e-14, atol=1e-14)
    rows = np.repeat(np.arange(31), np.diff(A.rowptr))
    ref = np.einsum("pk,pk->p", g[rows], x[A.col])
    np.testing.assert_allclose(oracle.sampled_product(A, g, x), ref, rtol=1e-14, atol=1e-14)


def _slice(A, nrows):
    """The first nrows rows of A with columns restricted to [0, nrows)."""
    rp, cols, vals = [0], [], []
    for i in range(nrows):
        seg = slice(A.rowptr[i], A.rowptr[i + 1])
        c = A.col[seg]
        m = c < nrows
        cols.append(c[m])
        vals.append(A.val[seg][m])
        rp.append(rp[-1] + int(m.sum()))
    return gen.CSR(nrows, nrows, np.array(rp, np.int64), np.concatenate(cols).astype(np.int32),
                   np.concatenate(vals))


def test_finite_differences_powerlaw_slice():
    full = gen.powerlaw(1 << 14, seed=gen.BASE_SEED + 3)
    A = _slice(full, 4096)
    w = 4
    x = gen.normal_block(A.nrows, w, 1)
    g = gen.normal_block(A.nrows, w, 2)
    h = 1e-6

    def loss(vals, xx):
        return float((g * oracle.spmmv(A, xx, val=vals)[0]).sum())

    dx = oracle.spmmv_transpose(A, g)
    dv = oracle.sampled_product(A, g, x)
    rng = np.random.default_rng(0)
    for j, k in zip(rng.integers(0, A.nrows, 12), rng.integers(0, w, 12)):
        xp, xm = x.copy(), x.copy()
        xp[j, k] += h
        xm[j, k] -= h
        fd = (loss(A.val, xp) - loss(A.val, xm)) / (2 * h)
        assert abs(fd - dx[j, k]) <= 1e-6 * (1 + abs(dx[j, k]))
    for p in rng.integers(0, A.nnz, 12):
        vp, vm = A.val.copy(), A.val.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss(vp, x) - loss(vm, x)) / (2 * h)
        assert abs(fd - dv[p]) <= 1e-6 * (1 + abs(dv[p]))


def test_cg_eigenvector_rhs():
    s = 24
    A = gen.laplace2d(s, 0.01)
    v = gen.laplace2d_mode(s, 2, 3)
    th = np.pi / (s + 1)
    lam = 4.01 - 2 * np.cos(2 * th) - 2 * np.cos(3 * th)
    X, its = oracle.cg(A, lam * v, tol=1e-12)
    np.testing.assert_allclose(X[:, 0], v, rtol=0, atol=1e-11)
    assert its[0] <= 3


def test_cg_against_direct_solver():
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    s = 20
    A = gen.laplace2d(s, 0.01)
    B = gen.block_vector(A.nrows, 3, 5)
    M = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, A.nrows))
    ref = spl.spsolve(M.tocsc(), B)
    X, _ = oracle.cg(A, B, tol=1e-12)
    kappa = 8.01 / 0.01
    np.testing.assert_allclose(X, ref, rtol=0, atol=kappa * 1e-12 * np.abs(ref).max())
    Xm, outer = oracle.mixed_precision_cg(A, B, tol=1e-10)
    r = B - oracle.spmmv(A, Xm)[0]
    assert np.all(np.linalg.norm(r, axis=0) <= 1e-10 * np.linalg.norm(B, axis=0))
    assert np.all(outer >= 2)  # float32 alone cannot reach 1e-10
    np.testing.assert_allclose(Xm, ref, rtol=0, atol=kappa * 1e-10 * np.abs(ref).max())
