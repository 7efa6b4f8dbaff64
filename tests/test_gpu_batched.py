"""Batched persistent SpMMV and mixed-precision CG on the GPU.

* every matrix's y against the oracle, entry by entry, at the tolerance of
  the single-matrix parity tests (tests/gpu_helpers.py: 1e-12 of the magnitude
  scale for float64, the float32 recursive-summation bound otherwise);
* every matrix of a batch gives exactly (bit for bit) the y of its solo
  sp_spmv run when both give each row one lane (C = 32): per row and column
  the products are then added in the same order whatever the lane layout;
  with rows split over several lanes the two agree within the tolerance;
* per-matrix dot products against the oracle within the derived dot bound;
* the CG solution: float64 residual <= 1e-10 ||b|| per column checked by the
  oracle's product, the closed-form solution for an eigenvector right-hand
  side, and the oracle's float64 CG solution within the conditioning bound;
* the 64-system workload at full size.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import assert_close, dot_bound, to_dev, tol_for
from tests.test_oracle_format import random_csr
from workloads import generators as gen

pytestmark = pytest.mark.gpu

DOTS = sellcs.SP_SPMV_DOT_YY | sellcs.SP_SPMV_DOT_XY | sellcs.SP_SPMV_DOT_XX


def _batch_inputs(seed, count, square=True):
    rng = np.random.default_rng(seed)
    mats, widths, Cs, sigmas = [], [], [], []
    for m in range(count):
        n = int(rng.integers(1, 3000))
        A = random_csr(n, n, float(rng.uniform(0.001, 0.02)), rng) if n > 1 else random_csr(1, 1, 1.0, rng)
        mats.append(A)
        widths.append(int(rng.integers(1, 9)))
        Cs.append(int(rng.choice([8, 16, 32])))
        sigmas.append(int(rng.choice([1, 32, 256, 1024])))
    return mats, widths, Cs, sigmas


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f32"), ("f32", "f64")])
def test_batched_equals_solo_and_oracle(cuda_ok, vdt, xdt):
    """Bit-equal to the solo run when both split rows over the same number of
    lanes (C = 32: one lane per row in both), within tolerance otherwise."""
    mats, widths, Cs, sigmas = _batch_inputs(1, 23)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    rng = np.random.default_rng(2)
    S = [sellcs.SellMatrix(A, C=C, sigma=s, dtype=vdt) for A, C, s in zip(mats, Cs, sigmas)]
    X = [rng.uniform(-1, 1, (A.ncols, w)) for A, w in zip(mats, widths)]
    Y0 = [rng.uniform(-1, 1, (A.nrows, w)) for A, w in zip(mats, widths)]
    if xdt == "f32":
        X = [a.astype(np.float32).astype(np.float64) for a in X]
        Y0 = [a.astype(np.float32).astype(np.float64) for a in Y0]
    xs = [to_dev(a, tdt) for a in X]
    y0s = [to_dev(a, tdt) for a in Y0]
    ys = [torch.full_like(a, float("nan")) for a in y0s]
    b = sellcs.Batch(S, widths, vec_dtype=xdt)
    b.bind(xs, ys, y0s)
    dots = torch.full((len(S) * 24,), float("nan"), dtype=torch.float64, device="cuda")
    flags = sellcs.SP_SPMV_SCALE | sellcs.SP_SPMV_AXPBY | DOTS
    b.spmv(flags, 0.5, -2.0, dots)
    torch.cuda.synchronize()
    d = dots.cpu().numpy().reshape(len(S), 3, 8)
    for m, (A, w) in enumerate(zip(mats, widths)):
        solo = y0s[m].clone()
        sellcs.spmv(S[m], xs[m], solo, alpha=0.5, beta=-2.0)
        torch.cuda.synchronize()
        yr, dr, _ = oracle.spmmv(A, X[m], val=oracle.round_values(A.val, vdt), alpha=0.5, beta=-2.0, y0=Y0[m],
                                 dot_yy=True, dot_xy=True, dot_xx=True)
        yg = ys[m].double().cpu().numpy()
        maxlen = int(np.diff(A.rowptr).max(initial=0))
        tol = tol_for(vdt, xdt, maxlen)
        sc = oracle.spmmv_scale(A, X[m], val=oracle.round_values(A.val, vdt), alpha=0.5, beta=-2.0, y0=Y0[m])
        if xdt == "f32":
            sc = sc + np.abs(yr)  # the float32 output rounds once more
        assert_close(yg, yr, sc, tol, f"batched y of matrix {m} vs oracle")
        if Cs[m] == 32:
            # one lane per row in both kernels: the same products added in the same order
            assert torch.equal(solo, ys[m]), f"matrix {m}: batched y differs from solo y"
        else:
            assert np.all(np.abs(solo.double().cpu().numpy() - yg) <= 2 * tol * sc + 1e-300)
        e = tol * sc
        for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
            assert_close(d[m, q, :w], dr[q * w:(q + 1) * w], dot_bound(name, yr, X[m], e, xdt, A.nrows), 1.0,
                         f"batched {name} of matrix {m}")
        assert np.all(np.isnan(d[m, :, w:])), "unused dot slots written"


def test_batched_cols_per_lane_choices(cuda_ok):
    mats, widths, Cs, sigmas = _batch_inputs(5, 6)
    widths = [8, 8, 4, 6, 2, 8]
    # C = 32: one lane per row, so every lane layout adds in the same order
    S = [sellcs.SellMatrix(A, C=32, sigma=s, dtype="f32") for A, s in zip(mats, sigmas)]
    rng = np.random.default_rng(3)
    xs = [to_dev(rng.uniform(-1, 1, (A.ncols, w)), torch.float32) for A, w in zip(mats, widths)]
    ref = None
    for cpl in ([1, 1, 1, 1, 1, 1], [2, 4, 2, 2, 2, 4], [4, 2, 4, 2, 1, 4], None):
        ys = [torch.zeros(A.nrows, w, dtype=torch.float32, device="cuda") for A, w in zip(mats, widths)]
        b = sellcs.Batch(S, widths, cols_per_lane=cpl, vec_dtype="f32")
        b.bind(xs, ys)
        b.spmv()
        torch.cuda.synchronize()
        if ref is None:
            ref = [y.clone() for y in ys]
        for y, r in zip(ys, ref):
            assert torch.equal(y, r)
    with pytest.raises(sellcs.SpError):
        sellcs.Batch(S, widths, cols_per_lane=[4, 4, 4, 4, 4, 4], vec_dtype="f32")  # 4 does not divide 6
    with pytest.raises(sellcs.SpError):
        sellcs.Batch(S, widths, cols_per_lane=[8, 1, 1, 1, 1, 1], vec_dtype="f32")  # above 4 floats per lane


def _cg_check(mats, Bs, Xg, tol=1e-10):
    for A, B, X in zip(mats, Bs, Xg):
        r = B - oracle.spmmv(A, X)[0]
        rel = np.linalg.norm(r, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(rel <= tol), rel


def test_cg_small_batch(cuda_ok):
    sides = [16, 23, 40, 7, 31, 64]
    widths = [1, 3, 8, 2, 5, 4]
    mats = [gen.laplace2d(s, 0.01) for s in sides]
    Bs = [gen.block_vector(A.nrows, w, 100 + i) for i, (A, w) in enumerate(zip(mats, widths))]
    S = [sellcs.SellMatrix(A, C=16, sigma=32) for A in mats]
    cg = sellcs.CG(S, widths)
    bs = [to_dev(B) for B in Bs]
    xs = [torch.zeros_like(b) for b in bs]
    for inner_f64 in (False, True):
        stats, rel = cg.solve(bs, xs, inner_f64=inner_f64)
        torch.cuda.synchronize()
        assert stats["converged"] == 1 and np.all(rel <= 1e-10), (stats, rel)
        if not inner_f64:
            assert stats["outer"] >= 2  # float32 alone cannot reach 1e-10
        Xg = [x.cpu().numpy() for x in xs]
        _cg_check(mats, Bs, Xg)
        kappa = 8.01 / 0.01
        for A, B, X in zip(mats, Bs, Xg):
            Xo, _ = oracle.cg(A, B, tol=1e-12)
            np.testing.assert_allclose(X, Xo, rtol=0, atol=kappa * 1e-10 * np.abs(Xo).max())


def test_cg_eigenvector_rhs(cuda_ok):
    s = 48
    A = gen.laplace2d(s, 0.01)
    th = np.pi / (s + 1)
    modes = [(1, 1), (3, 7), (48, 48)]
    V = np.stack([gen.laplace2d_mode(s, p, q) for p, q in modes], axis=1)
    lam = np.array([4.01 - 2 * np.cos(p * th) - 2 * np.cos(q * th) for p, q in modes])
    cg = sellcs.CG([sellcs.SellMatrix(A, C=32, sigma=1)], [3])
    b = to_dev(V * lam[None, :])
    x = torch.zeros_like(b)
    stats, rel = cg.solve([b], [x])
    assert stats["converged"] == 1
    np.testing.assert_allclose(x.cpu().numpy(), V, rtol=0, atol=1e-9)


@pytest.mark.slow
def test_cg_batch_full_size(cuda_ok):
    """64 systems L_2D(s) + 0.01 I, s in [64, 512], widths 1..8 (about 6.4M
    rows in all): every column reaches ||b - A x|| <= 1e-10 ||b||."""
    batch = gen.workload_cg_batch()
    mats = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    widths = [B.shape[1] for B in Bs]
    S = [sellcs.SellMatrix(A, C=32, sigma=1) for A in mats]
    cg = sellcs.CG(S, widths)
    bs = [to_dev(B) for B in Bs]
    xs = [torch.zeros_like(b) for b in bs]
    stats, rel = cg.solve(bs, xs)
    torch.cuda.synchronize()
    assert stats["converged"] == 1, stats
    _cg_check(mats, Bs, [x.cpu().numpy() for x in xs])
