"""Shared helpers of the GPU parity tests: run one augmented product through the
C ABI and the same product through the oracle, and compare them with the
tolerance the arithmetic allows.

Tolerance (derived, stated once here): a row sum of n products accumulated
recursively in a format with unit roundoff u is off by at most
gamma_n = n u / (1 - n u) times sum |a_ij x_j| (Higham, Accuracy and Stability
of Numerical Algorithms, Sec. 3.1); the epilogue adds at most four more
roundings, and widening x from float64 to float32 before the product one more.
So, per entry, |y_gpu - y| <= tol * s with s = |alpha|(|A||x|) +
|alpha gamma||x| + |beta||y0| and

    tol = 1e-12                         values and vectors float64 (the stated target)
    tol = 1.1 (n_max + 6) 2^-24         float32 row sums (f32 or bf16 values)

where the oracle is given exactly the values the GPU stores (rounded to f32 or
bf16), so the storage rounding is not part of this comparison and is reported
separately against the unrounded float64 matrix.

Dot products (dot_bound): the GPU sums terms of its own y, so its result D^
differs from the oracle's D (terms of the oracle's y) by
  (1) the propagated error of y: with e_i = tol * s_i the bound on |y^_i - y_i|,
      |sum y^_i^2 - sum y_i^2| <= sum e_i (2|y_i| + e_i) and
      |sum x_i y^_i - sum x_i y_i| <= sum |x_i| e_i  (x is exact on both sides);
  (2) the accumulation error: a sum in which every term passes through at most
      n additions in a format of unit roundoff u is off by at most
      gamma_n = n u / (1 - n u) times the sum of the terms' magnitudes.  Float32
      vectors add in float over at most SP_DOT_RUN_F32 rows per lane plus a
      float tree of at most 5 levels (n = SP_DOT_RUN_F32 + 5, u = 2^-24); every
      later stage (per-warp bank, warp tree, block, grid) adds in float64, and
      no term passes through more than N + 2100 of those (u = 2^-53).
"""
import numpy as np
import torch

import oracle
from paper_1507_08101_gb300 import sellcs

U32 = 2.0 ** -24


def tol_for(vdt: str, xdt: str, maxlen: int) -> float:
    if vdt == "f64" and xdt == "f64":
        return 1e-12
    return 1.1 * (maxlen + 6) * U32


U53 = 2.0 ** -53


def gamma(n, u):
    return n * u / (1 - n * u)


def dot_bound(name, yr, X, e, xdt, N):
    """Bound on |dot_gpu - dot_oracle| per column (derivation in the module
    docstring).  yr: oracle y (N x w), X: x as both sides use it, e: per-entry
    bound on |y_gpu - y_oracle| (N x w)."""
    g = gamma(N + 2100, U53) + 1e-15  # float64 stages + the oracle's own rounding
    if xdt == "f32":
        g += gamma(sellcs.SP_DOT_RUN_F32 + 5, U32)
    xa = np.abs(X[:N])
    if name == "dot_yy":
        prop = e * (2 * np.abs(yr) + e)
        terms = yr * yr + prop
    elif name == "dot_xy":
        prop = xa * e
        terms = xa * (np.abs(yr) + e)
    else:
        prop = np.zeros_like(xa)
        terms = xa * xa
    return prop.sum(0) + g * terms.sum(0)


def to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def assert_close(got, ref, scale, tol, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    bound = tol * np.asarray(scale) + 1e-300
    bad = err > bound
    if bad.any():
        idx = np.argwhere(bad)[:5]
        ratio = float(np.max(err / bound))
        raise AssertionError(f"{what}: {int(bad.sum())} entries beyond tol {tol:g} (worst err/bound {ratio:.3g}); "
                             f"first {idx.tolist()} got {got[bad][:5]} ref {ref[bad][:5]}")


def run_case(A, C, sigma, w, flags, *, vdt="f64", xdt="f64", layout="row", ld_pad=0, seed=0, alpha=0.7,
             beta=-1.3, gamma_s=0.25, delta=0.9, eta=0.1, mat=None):
    """One augmented product on the GPU and in the oracle; asserts parity.

    flags: set of names among scale, shift, vshift, axpby, dot_yy, dot_xy,
    dot_xx, chain.  Returns (y_gpu, y_ref) for further checks."""
    rng = np.random.default_rng(seed)
    N, M = A.nrows, A.ncols
    X = rng.uniform(-1, 1, (M, w))
    Y0 = rng.uniform(-1, 1, (N, w))
    Z0 = rng.uniform(-1, 1, (N, w))
    gv = rng.uniform(-1, 1, w)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    if xdt == "f32":
        X, Y0, Z0 = (a.astype(np.float32).astype(np.float64) for a in (X, Y0, Z0))
    vals_stored = oracle.round_values(A.val, vdt)
    if mat is None:
        mat = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=vdt)

    def dev_block(a, n):
        if layout == "row":
            base = torch.full((n, w + ld_pad), float("nan"), dtype=tdt, device="cuda")
            base[:, :w] = to_dev(a, tdt)
            return base, base[:, :w]
        base = torch.full((w + ld_pad, n), float("nan"), dtype=tdt, device="cuda")
        base[:w, :] = to_dev(a.T, tdt)
        return base, base[:w, :].t()

    xb, xv = dev_block(X, M)
    yb, yv = dev_block(Y0 if "axpby" in flags else np.full((N, w), np.nan), N)
    zb, zv = dev_block(Z0, N)
    dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device="cuda")
    gamma = gamma_s if "shift" in flags else (gv if "vshift" in flags else None)
    lay = sellcs.SP_ROW_MAJOR if layout == "row" else sellcs.SP_COL_MAJOR
    if w == 1 and ld_pad == 0:
        # exercise 1-D views too
        xv, yv, zv = xv[:, 0], yv[:, 0], zv[:, 0]
    sellcs.spmv(mat, xv, yv, alpha=alpha if "scale" in flags else None, gamma=gamma,
                beta=beta if "axpby" in flags else None, dot_yy="dot_yy" in flags, dot_xy="dot_xy" in flags,
                dot_xx="dot_xx" in flags, z=zv if "chain" in flags else None,
                delta=delta if "chain" in flags else None, eta=eta if "chain" in flags else None,
                dot=dot, layout=lay)
    torch.cuda.synchronize()
    y = yv.reshape(N, w).double().cpu().numpy()
    z = zv.reshape(N, w).double().cpu().numpy()
    d = dot.cpu().numpy()

    yr, dr, zr = oracle.spmmv(A, X, val=vals_stored, alpha=alpha if "scale" in flags else None, gamma=gamma,
                              beta=beta if "axpby" in flags else None, y0=Y0 if "axpby" in flags else None,
                              dot_yy="dot_yy" in flags, dot_xy="dot_xy" in flags, dot_xx="dot_xx" in flags,
                              delta=delta if "chain" in flags else None, eta=eta if "chain" in flags else None,
                              z0=Z0 if "chain" in flags else None)
    s = oracle.spmmv_scale(A, X, val=vals_stored, alpha=alpha if "scale" in flags else None, gamma=gamma,
                           beta=beta if "axpby" in flags else None, y0=Y0 if "axpby" in flags else None)
    maxlen = int(np.diff(A.rowptr).max(initial=0))
    tol = tol_for(vdt, xdt, maxlen)
    # float32 output vectors round the result once more
    if xdt == "f32":
        s = s + np.abs(yr)
    assert_close(y, yr, s, tol, f"y C={C} sigma={sigma} w={w} {sorted(flags)} {vdt}/{xdt} {layout}")
    # columns beyond w (ld padding) untouched
    if ld_pad:
        pad = (yb[:, w:] if layout == "row" else yb[w:, :]).cpu().numpy()
        assert np.all(np.isnan(pad)), "padding columns of y were written"
    if "chain" in flags:
        sz = 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + s)
        assert_close(z, zr, sz, tol + (U32 if xdt == "f32" else 0), "z")
    # dots: against the oracle within dot_bound, and unrequested slots untouched
    e = tol * s
    for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
        got = d[q * w:(q + 1) * w]
        if name in flags:
            assert_close(got, dr[q * w:(q + 1) * w], dot_bound(name, yr, X, e, xdt, N), 1.0, name)
        else:
            assert np.all(np.isnan(got)), f"{name} slot written though not requested"
    return y, yr, mat
