"""Oracle for the SELL-C-sigma augmented SpMMV -- TEST INFRASTRUCTURE ONLY.

Plain double-precision CPU code (``sell_oracle.c`` through ctypes, plus numpy
for the iterative drivers).  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the library under test never
does, and this package imports nothing from it.

Functions and the passage of GHOST (arxiv 1507.08101) each one follows:

* :func:`sell_from_csr`, :func:`sell_to_csr` -- SELL-C-sigma storage (Sec.
  "Sparse matrix storage": chunks of C rows, zero padding to the chunk's longest
  row, column-wise chunk storage, sigma-window sort by nonzero count).
* :func:`spmmv` -- the augmented product y = alpha (A - gamma I) x + beta y with
  <y,y>, <x,y>, <x,x> and z = delta z + eta y (Sec. "Kernel fusion").
* :func:`spmmv_transpose`, :func:`sampled_product` -- derivatives of y = A x.
* :func:`cg` -- conjugate gradients, one column at a time (the CG sample
  application of Sec. "Introduction"); :func:`mixed_precision_cg` -- iterative
  refinement around a float32 inner solve.
* :func:`round_values` -- float32 and bfloat16 storage rounding.
* :func:`tsmttsm`, :func:`tsmm` -- the tall and skinny block-vector kernels of
  the dense-matrix section (X <- alpha V^T W + beta X, W <- alpha V X + beta W),
  by their definition with numpy's matrix product.
* :func:`kpm_moments` -- Chebyshev moments mu_k = <x, T_k(A~) x> of the kernel
  polynomial method that Sec. "Kernel fusion" names as the solver the fused
  product serves (A. Weisse, G. Wellein, A. Alvermann and H. Fehske, "The
  kernel polynomial method", Rev. Mod. Phys. 78 (2006)), by the definition:
  the three-term recurrence up to k and one inner product per moment.

Pins (tests/test_oracle_*.py) tie every function to something other than
itself: dense brute force, closed-form eigenpairs, format identities from the
paper, finite differences and a library direct solver.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sell_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle's C part with gcc (plain -O2, no fast-math)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c99",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_LIBDIR, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False):
    """The same C source with OpenMP (-fopenmp), for the all-cores timing
    baseline (orc_spmmv_omp).  Returns the library path, or None when the
    compiler cannot build it."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".{os.getpid()}.tmp"
        try:
            subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c99", "-fopenmp",
                                   "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"], stderr=subprocess.DEVNULL)
        except (OSError, subprocess.CalledProcessError):
            return None
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load_omp():
    global _lib_omp
    if _lib_omp is None:
        if build_omp() is None:
            return None
        L = ct.CDLL(_LIB_OMP)
        P, I64, I, D = ct.c_void_p, ct.c_int64, ct.c_int, ct.c_double
        L.orc_spmmv_omp.restype = None
        L.orc_spmmv_omp.argtypes = [I64, P, P, P, I, P, I64, P, I64, P, I64,
                                    I, D, I, P, I, D, I, I, I, P, I, D, D, P, I64, I]
        _lib_omp = L
    return _lib_omp


def spmmv_omp(A, x, *, nthreads, alpha=None, gamma=None, beta=None, y0=None, dot_yy=False, dot_xy=False,
              dot_xx=False, delta=None, eta=None, z0=None):
    """spmmv with the rows shared among ``nthreads`` OpenMP threads (timing
    baseline only; see orc_spmmv_omp).  Same return values as spmmv; None if
    OpenMP is not available."""
    lib = _load_omp()
    if lib is None:
        return None
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    x = _c(x, np.float64)
    N, w = A.nrows, x.shape[1]
    y = np.empty((N, w), np.float64)
    g = np.zeros(w) if gamma is None else np.broadcast_to(np.asarray(gamma, np.float64), (w,)).copy()
    do_axpby = beta is not None
    y0c = _c(y0, np.float64).reshape(N, w) if do_axpby else np.zeros((1, 1))
    do_chain = z0 is not None
    z = _c(z0, np.float64).reshape(N, w).copy() if do_chain else np.zeros((1, 1))
    dot = np.full(3 * w, np.nan)
    lib.orc_spmmv_omp(N, _p(_c(A.rowptr, np.int64)), _p(_c(A.col, np.int32)), _p(_c(A.val, np.float64)), w,
                      _p(x), w, _p(y), w, _p(y0c), w,
                      int(alpha is not None), float(alpha if alpha is not None else 1.0),
                      int(gamma is not None), _p(g), int(do_axpby), float(beta if do_axpby else 0.0),
                      int(dot_yy), int(dot_xy), int(dot_xx), _p(dot),
                      int(do_chain), float(delta if do_chain else 0.0), float(eta if do_chain else 0.0),
                      _p(z), w, int(nthreads))
    return y, dot, (z if do_chain else None)


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ct.CDLL(_LIB)
        P = ct.c_void_p
        I64 = ct.c_int64
        I = ct.c_int
        D = ct.c_double
        _lib.orc_sell_structure.restype = I64
        _lib.orc_sell_structure.argtypes = [I64, P, I, I64, P, P, P, P]
        _lib.orc_sell_fill.restype = None
        _lib.orc_sell_fill.argtypes = [I64, P, P, P, I, P, P, P, P, P]
        _lib.orc_sell_to_csr.restype = None
        _lib.orc_sell_to_csr.argtypes = [I64, I, P, P, P, P, P, P, P, P]
        _lib.orc_spmmv.restype = None
        _lib.orc_spmmv.argtypes = [I64, I64, P, P, P, I, P, I64, P, I64, P, I64,
                                   I, D, I, P, I, D, I, I, I, P, I, D, D, P, I64]
        _lib.orc_spmmv_scale.restype = None
        _lib.orc_spmmv_scale.argtypes = [I64, P, P, P, I, P, I64, P, I64, D, P, D, I, P, I64]
        _lib.orc_spmmv_transpose.restype = None
        _lib.orc_spmmv_transpose.argtypes = [I64, I64, P, P, P, I, P, P]
        _lib.orc_sampled_product.restype = None
        _lib.orc_sampled_product.argtypes = [I64, P, P, I, P, P, P]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------- storage format

@dataclass
class SellRef:
    """SELL-C-sigma arrays as the oracle builds them (all host numpy)."""
    nrows: int
    C: int
    sigma: int
    perm: np.ndarray  # int32, nch*C: slot -> original row (-1 = padding row)
    slotlen: np.ndarray  # int32, nch*C
    chunklen: np.ndarray  # int32, nch
    chunkptr: np.ndarray  # int64, nch+1
    col: np.ndarray  # int32, nstored
    val: np.ndarray  # float64, nstored

    @property
    def nchunks(self) -> int:
        return int(self.chunklen.size)

    @property
    def nstored(self) -> int:
        return int(self.chunkptr[-1])


def sell_from_csr(A, C: int, sigma: int) -> SellRef:
    """CSR -> SELL-C-sigma (sorted windows of sigma rows, chunks of C rows)."""
    lib = _load()
    N = A.nrows
    assert C >= 1 and sigma >= 1
    nch = (N + C - 1) // C
    rowptr = _c(A.rowptr, np.int64)
    perm = np.empty(nch * C, np.int32)
    slotlen = np.empty(nch * C, np.int32)
    chunklen = np.empty(nch, np.int32)
    chunkptr = np.empty(nch + 1, np.int64)
    nst = lib.orc_sell_structure(N, _p(rowptr), C, sigma, _p(perm), _p(slotlen), _p(chunklen), _p(chunkptr))
    col = np.empty(max(nst, 1), np.int32)[:nst]
    val = np.empty(max(nst, 1), np.float64)[:nst]
    colc = _c(A.col, np.int32)
    valc = _c(A.val, np.float64)
    lib.orc_sell_fill(N, _p(rowptr), _p(colc), _p(valc), C, _p(perm), _p(chunklen), _p(chunkptr),
                      _p(col), _p(val))
    return SellRef(N, C, sigma, perm, slotlen, chunklen, chunkptr, col, val)


def sell_to_csr(S: SellRef):
    """SELL-C-sigma -> (rowptr, col, val) in the original row order."""
    lib = _load()
    nnz = int(S.slotlen.astype(np.int64).sum())
    rowptr = np.empty(S.nrows + 1, np.int64)
    col = np.empty(max(nnz, 1), np.int32)[:nnz]
    val = np.empty(max(nnz, 1), np.float64)[:nnz]
    lib.orc_sell_to_csr(S.nrows, S.C, _p(_c(S.perm, np.int32)), _p(_c(S.slotlen, np.int32)),
                        _p(_c(S.chunkptr, np.int64)), _p(_c(S.col, np.int32)), _p(_c(S.val, np.float64)),
                        _p(rowptr), _p(col), _p(val))
    return rowptr, col, val


# --------------------------------------------------------------------------- augmented product

def spmmv(A, x, *, alpha=None, gamma=None, beta=None, y0=None, dot_yy=False, dot_xy=False, dot_xx=False,
          delta=None, eta=None, z0=None, val=None):
    """Augmented SpMMV on CSR in float64.

    ``alpha`` None = no scaling; ``gamma`` None = no shift, a scalar = one
    shift for all columns, a sequence = one shift per column; ``beta`` None =
    y0 not used.  ``delta``/``eta`` with ``z0`` turn on z = delta z0 + eta y.
    ``val`` overrides A's values (e.g. values rounded to a storage precision).
    Returns (y, dot[3w], z) -- dot slots that were not requested are NaN, z is
    None without the chain.
    """
    lib = _load()
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    x = _c(x, np.float64)
    N, w = A.nrows, x.shape[1]
    assert x.shape[0] == A.ncols
    vals = _c(A.val if val is None else val, np.float64)
    y = np.empty((N, w), np.float64)
    if gamma is None:
        g = np.zeros(w)
    else:
        g = np.broadcast_to(np.asarray(gamma, np.float64), (w,)).copy()
    do_axpby = beta is not None
    y0c = _c(y0, np.float64).reshape(N, w) if do_axpby else np.zeros((1, 1))
    do_chain = z0 is not None
    z = _c(z0, np.float64).reshape(N, w).copy() if do_chain else np.zeros((1, 1))
    dot = np.full(3 * w, np.nan)
    lib.orc_spmmv(N, A.ncols, _p(_c(A.rowptr, np.int64)), _p(_c(A.col, np.int32)), _p(vals), w,
                  _p(x), w, _p(y), w, _p(y0c), w,
                  int(alpha is not None), float(alpha if alpha is not None else 1.0),
                  int(gamma is not None), _p(g), int(do_axpby), float(beta if do_axpby else 0.0),
                  int(dot_yy), int(dot_xy), int(dot_xx), _p(dot),
                  int(do_chain), float(delta if do_chain else 0.0), float(eta if do_chain else 0.0),
                  _p(z), w)
    return y, dot, (z if do_chain else None)


def spmmv_scale(A, x, *, alpha=None, gamma=None, beta=None, y0=None, val=None):
    """Entry-wise magnitude |alpha| (|A||x|) + |alpha gamma||x| + |beta||y0| used
    to express a rounding error of the augmented product relative to its terms."""
    lib = _load()
    x = np.asarray(x, np.float64)
    if x.ndim == 1:
        x = x[:, None]
    x = _c(x, np.float64)
    N, w = A.nrows, x.shape[1]
    vals = _c(A.val if val is None else val, np.float64)
    g = np.zeros(w) if gamma is None else np.broadcast_to(np.asarray(gamma, np.float64), (w,)).copy()
    use_y0 = beta is not None
    y0c = _c(y0, np.float64).reshape(N, w) if use_y0 else np.zeros((1, 1))
    s = np.empty((N, w))
    lib.orc_spmmv_scale(N, _p(_c(A.rowptr, np.int64)), _p(_c(A.col, np.int32)), _p(vals), w, _p(x), w,
                        _p(y0c), w, float(1.0 if alpha is None else alpha), _p(g),
                        float(beta if use_y0 else 0.0), int(use_y0), _p(s), w)
    return s


def spmmv_transpose(A, g, val=None):
    """dx = A^T g (ncols x w)."""
    lib = _load()
    g = np.asarray(g, np.float64)
    if g.ndim == 1:
        g = g[:, None]
    g = _c(g, np.float64)
    w = g.shape[1]
    dx = np.empty((A.ncols, w))
    vals = _c(A.val if val is None else val, np.float64)
    lib.orc_spmmv_transpose(A.nrows, A.ncols, _p(_c(A.rowptr, np.int64)), _p(_c(A.col, np.int32)),
                            _p(vals), w, _p(g), _p(dx))
    return dx


def sampled_product(A, g, x):
    """dvals[p] = sum_k g[row(p), k] x[col(p), k] for every nonzero p (CSR order)."""
    lib = _load()
    g = _c(np.asarray(g, np.float64).reshape(A.nrows, -1), np.float64)
    x = _c(np.asarray(x, np.float64).reshape(A.ncols, -1), np.float64)
    w = g.shape[1]
    out = np.empty(A.nnz)
    lib.orc_sampled_product(A.nrows, _p(_c(A.rowptr, np.int64)), _p(_c(A.col, np.int32)), w, _p(g), _p(x),
                            _p(out))
    return out


# --------------------------------------------------------------------------- storage precision

def round_values(v, dtype: str) -> np.ndarray:
    """Round float64 values to a storage precision and return them as float64.

    ``"f64"`` unchanged; ``"f32"`` IEEE round-to-nearest-even; ``"bf16"``
    round to float32 first, then keep the top 16 bits of the float32 with
    round-to-nearest-even on the 16 dropped bits (the definition of bfloat16
    rounding), NaN kept as a quiet NaN.
    """
    v = np.asarray(v, np.float64)
    if dtype == "f64":
        return v.copy()
    f = v.astype(np.float32)
    if dtype == "f32":
        return f.astype(np.float64)
    assert dtype == "bf16"
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(f)
    r = np.where(nan, (u | 0x00400000) & 0xFFFF0000, r)
    return (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------- solvers

def cg(A, B, tol: float = 1e-10, maxit: int = 10000, x0=None):
    """Conjugate gradients in float64, each column of B on its own.

    Stops a column when ||b - A x|| <= tol ||b|| (recursive residual), then
    returns X and the iteration counts.
    """
    B = np.asarray(B, np.float64)
    if B.ndim == 1:
        B = B[:, None]
    N, w = B.shape
    X = np.zeros((N, w)) if x0 is None else np.array(x0, np.float64).reshape(N, w)
    its = np.zeros(w, np.int64)
    for k in range(w):
        b = B[:, k].copy()
        x = X[:, k].copy()
        r = b - spmmv(A, x)[0][:, 0]
        p = r.copy()
        rr = float(r @ r)
        bn = float(np.sqrt(b @ b))
        it = 0
        while np.sqrt(rr) > tol * bn and it < maxit:
            q = spmmv(A, p)[0][:, 0]
            a = rr / float(p @ q)
            x += a * p
            r -= a * q
            rr_new = float(r @ r)
            p = r + (rr_new / rr) * p
            rr = rr_new
            it += 1
        X[:, k] = x
        its[k] = it
    return X, its


def mixed_precision_cg(A, B, tol: float = 1e-10, inner_tol: float = 1e-4, max_outer: int = 50,
                       inner_maxit: int = 10000):
    """Iterative refinement: float64 residual r = b - A x, a float32 CG solve of
    A d = r to relative tolerance ``inner_tol`` (values and vectors rounded to
    float32, float32 arithmetic), float64 update x += d; until
    ||b - A x|| <= tol ||b|| per column.  Returns X and outer-step counts."""
    B = np.asarray(B, np.float64)
    if B.ndim == 1:
        B = B[:, None]
    N, w = B.shape
    A32 = np.float32
    v32 = A.val.astype(A32)
    X = np.zeros((N, w))
    outer = np.zeros(w, np.int64)
    for k in range(w):
        b = B[:, k]
        bn = np.sqrt(b @ b)
        x = np.zeros(N)
        for o in range(max_outer):
            r = b - spmmv(A, x)[0][:, 0]
            if np.sqrt(r @ r) <= tol * bn:
                break
            outer[k] = o + 1
            r32 = r.astype(A32)
            d = np.zeros(N, A32)
            rr32 = r32.copy()
            p = rr32.copy()
            rho = A32(rr32 @ rr32)
            r0 = np.sqrt(rho)
            for _ in range(inner_maxit):
                if np.sqrt(rho) <= inner_tol * r0:
                    break
                q = _spmv_f32(A, v32, p)
                a = A32(rho / A32(p @ q))
                d = (d + a * p).astype(A32)
                rr32 = (rr32 - a * q).astype(A32)
                rho_new = A32(rr32 @ rr32)
                p = (rr32 + A32(rho_new / rho) * p).astype(A32)
                rho = rho_new
            x = x + d.astype(np.float64)
        X[:, k] = x
    return X, outer


def _spmv_f32(A, v32, p):
    """Row sums of float32 products in float32 (plain loop order of CSR rows)."""
    prod = (v32 * p[A.col]).astype(np.float32)
    return np.add.reduceat(prod, A.rowptr[:-1]).astype(np.float32) * (np.diff(A.rowptr) > 0)


# --------------------------------------------------------------------------- KPM moments

def kpm_moments(A, X, nmom: int, a: float, b: float):
    """mu[k, c] = <x_c, T_k(A~) x_c> for k < nmom, A~ = (A - b I) / a.

    The definition itself: w_0 = x, w_1 = A~ w_0, w_{k+1} = 2 A~ w_k - w_{k-1}
    (the Chebyshev recurrence), and mu_k = <w_0, w_k>, one product per k.
    Returns an (nmom, w) float64 array."""
    X = np.asarray(X, np.float64)
    if X.ndim == 1:
        X = X[:, None]
    w0 = X.copy()
    mu = np.empty((nmom, X.shape[1]))
    mu[0] = (w0 * w0).sum(0)
    if nmom == 1:
        return mu
    w1 = (spmmv(A, w0)[0] - b * w0) / a
    mu[1] = (w0 * w1).sum(0)
    prev, cur = w0, w1
    for k in range(2, nmom):
        nxt = 2.0 * (spmmv(A, cur)[0] - b * cur) / a - prev
        mu[k] = (w0 * nxt).sum(0)
        prev, cur = cur, nxt
    return mu


# --------------------------------------------------------------------------- tall and skinny kernels

def tsmttsm(V, W, X0=None, alpha=1.0, beta=0.0):
    """alpha V^T W + beta X0 in float64."""
    V = np.asarray(V, np.float64)
    W = np.asarray(W, np.float64)
    out = alpha * (V.T @ W)
    if beta != 0.0:
        out = out + beta * np.asarray(X0, np.float64)
    return out


def tsmm(V, X, W0=None, alpha=1.0, beta=0.0):
    """alpha V X + beta W0 in float64."""
    out = alpha * (np.asarray(V, np.float64) @ np.asarray(X, np.float64))
    if beta != 0.0:
        out = out + beta * np.asarray(W0, np.float64)
    return out

