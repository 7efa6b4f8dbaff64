"""Seeded synthetic CSR matrices and block vectors shaped like the paper's workloads.

These stand in for the SuiteSparse matrices the paper measures on (ML_Geer,
cage15, 3Dspectralwave), which are not available here; no dataset content is
reproduced.  All five workloads are built from closed structural recipes and
the counter-based streams of :mod:`workloads.rng`:

* ``laplace3d``      3D 7-point Dirichlet Laplacian (diag 6, off-diagonal -1),
                     natural lexicographic order.
* ``irregular_band`` rows of uniform random length, 90 % of columns in a
                     +-band around the diagonal and 10 % uniform.
* ``anderson3d``     3D periodic tight-binding lattice with on-site disorder
                     uniform in [-W/2, W/2] (Anderson model), the matrix of the
                     kernel polynomial / Chebyshev workloads.
* ``powerlaw``       row lengths from a discrete power law, uniform columns.
* ``laplace2d``      2D 5-point Dirichlet Laplacian plus a diagonal shift
                     (SPD; the CG workload), in batches of uneven size.

Every matrix comes out in canonical CSR: int64 row pointers, int32 column
indices sorted ascending inside each row and free of duplicates, float64 values.
Nothing here multiplies a matrix by a vector: this module only makes inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import rng

BASE_SEED = 20150729

# stream tags (arbitrary distinct integers)
_T_ROWLEN, _T_KIND, _T_BAND, _T_UNI, _T_VAL, _T_X, _T_DIAG, _T_SIZE, _T_W, _T_RHS = range(1, 11)


@dataclass
class CSR:
    nrows: int
    ncols: int
    rowptr: np.ndarray  # int64, nrows + 1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr)


def _finish(nrows, ncols, rowptr, col, val, **meta) -> CSR:
    return CSR(int(nrows), int(ncols), np.ascontiguousarray(rowptr, dtype=np.int64),
               np.ascontiguousarray(col, dtype=np.int32), np.ascontiguousarray(val, dtype=np.float64),
               dict(meta))


# --------------------------------------------------------------------------- stencils

def laplace3d(n: int = 32) -> CSR:
    """3D 7-point Laplacian on an n^3 grid with Dirichlet boundaries.

    Row index of grid point (i, j, k) is i + n*(j + n*k); diagonal 6, each
    existing neighbour -1.  n=32 gives N=32,768 and nnz=223,232.
    """
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    i = idx % n
    j = (idx // n) % n
    k = idx // (n * n)
    # candidate neighbours in ascending column order
    offs = [(-n * n, k > 0), (-n, j > 0), (-1, i > 0), (0, np.ones(N, bool)),
            (1, i < n - 1), (n, j < n - 1), (n * n, k < n - 1)]
    cols = np.stack([idx + o for o, _ in offs], axis=1)
    mask = np.stack([m for _, m in offs], axis=1)
    vals = np.where(np.arange(7) == 3, 6.0, -1.0)[None, :].repeat(N, 0)
    rowlen = mask.sum(1)
    rowptr = np.zeros(N + 1, np.int64)
    np.cumsum(rowlen, out=rowptr[1:])
    return _finish(N, N, rowptr, cols[mask], vals[mask], kind="laplace3d", n=n)


def laplace2d(s: int, shift: float = 0.01) -> CSR:
    """2D 5-point Dirichlet Laplacian on an s^2 grid plus ``shift`` on the diagonal.

    Row of grid point (i, j) is i + s*j; diagonal 4 + shift, neighbours -1.
    """
    N = s * s
    idx = np.arange(N, dtype=np.int64)
    i = idx % s
    j = idx // s
    offs = [(-s, j > 0), (-1, i > 0), (0, np.ones(N, bool)), (1, i < s - 1), (s, j < s - 1)]
    cols = np.stack([idx + o for o, _ in offs], axis=1)
    mask = np.stack([m for _, m in offs], axis=1)
    vals = np.where(np.arange(5) == 2, 4.0 + shift, -1.0)[None, :].repeat(N, 0)
    rowlen = mask.sum(1)
    rowptr = np.zeros(N + 1, np.int64)
    np.cumsum(rowlen, out=rowptr[1:])
    return _finish(N, N, rowptr, cols[mask], vals[mask], kind="laplace2d", s=s, shift=shift)


def anderson3d(n: int = 128, W: float = 16.5, seed: int = BASE_SEED + 2, disorder: bool = True) -> CSR:
    """3D Anderson model on an n^3 periodic lattice: hopping -1 to the six
    neighbours (with wrap-around), on-site energy uniform in [-W/2, W/2].

    ``disorder=False`` sets the diagonal to zero (a clean periodic lattice whose
    eigenvectors are plane waves).  Needs n >= 3 so that the six neighbours are
    distinct.
    """
    assert n >= 3
    N = n ** 3
    idx = np.arange(N, dtype=np.int64)
    i = idx % n
    j = (idx // n) % n
    k = idx // (n * n)

    def at(ii, jj, kk):
        return (ii % n) + n * ((jj % n) + n * (kk % n))

    cols = np.stack([at(i, j, k - 1), at(i, j - 1, k), at(i - 1, j, k), idx,
                     at(i + 1, j, k), at(i, j + 1, k), at(i, j, k + 1)], axis=1)
    if disorder:
        diag = rng.uniform(rng.stream_key(seed, _T_DIAG), idx, -W / 2, W / 2)
    else:
        diag = np.zeros(N)
    vals = np.full((N, 7), -1.0)
    vals[:, 3] = diag
    order = np.argsort(cols, axis=1, kind="stable")
    cols = np.take_along_axis(cols, order, 1)
    vals = np.take_along_axis(vals, order, 1)
    rowptr = np.arange(0, 7 * N + 1, 7, dtype=np.int64)
    return _finish(N, N, rowptr, cols.ravel(), vals.ravel(), kind="anderson3d", n=n, W=W,
                   disorder=disorder)


# --------------------------------------------------------------------------- random patterns

def _rows_of(rowptr: np.ndarray, rows: np.ndarray):
    """Entry indices and owning rows of all entries of the given rows."""
    lens = rowptr[rows + 1] - rowptr[rows]
    starts = rowptr[rows]
    own = np.repeat(rows, lens)
    first = np.repeat(np.cumsum(lens) - lens, lens)
    ent = np.repeat(starts, lens) + (np.arange(own.size, dtype=np.int64) - first)
    return ent, own


def _random_pattern(N: int, ncols: int, rowlen: np.ndarray, draw, lmax: int):
    """Draw distinct columns for every row.

    ``draw(ent, own, attempt)`` proposes a column for each entry index; a
    proposal outside [0, ncols) or equal to the column of a lower-numbered entry
    of the same row is redrawn with the next attempt number until none is left.
    Columns are then sorted ascending in each row.
    """
    rowptr = np.zeros(N + 1, np.int64)
    np.cumsum(rowlen, out=rowptr[1:])
    nnz = int(rowptr[-1])
    own_all = np.repeat(np.arange(N, dtype=np.int64), rowlen)
    col = np.full(nnz, -1, np.int64)
    cb = max(1, int(ncols - 1).bit_length())
    sb = max(1, int(lmax - 1).bit_length())
    assert int(N - 1).bit_length() + cb + sb <= 63
    pending = np.arange(nnz, dtype=np.int64)
    attempt = 0
    while pending.size:
        col[pending] = draw(pending, own_all[pending], attempt)
        rows = np.unique(own_all[pending])
        ent, own = _rows_of(rowptr, rows)
        c = col[ent]
        bad = (c < 0) | (c >= ncols)
        slot = ent - rowptr[own]
        key = (own << (cb + sb)) | (np.clip(c, 0, ncols - 1) << sb) | slot
        key = np.where(bad, -1, key)
        ks = np.sort(key)
        ks = ks[ks >= 0]
        dup_mask = np.zeros(ks.size, bool)
        dup_mask[1:] = (ks[1:] >> sb) == (ks[:-1] >> sb)
        dup = ks[dup_mask]
        dup_ent = rowptr[dup >> (cb + sb)] + (dup & ((1 << sb) - 1))
        pending = np.union1d(ent[bad], dup_ent)
        attempt += 1
        if attempt > 1000:
            raise RuntimeError("column draw did not converge")
    key = np.sort((own_all << cb) | col)
    col = key & ((1 << cb) - 1)
    return rowptr, col


def irregular_band(N: int = 1 << 21, lmin: int = 4, lmax: int = 64, band: int = 4096,
                   p_band: float = 0.9, seed: int = BASE_SEED + 1) -> CSR:
    """Irregular random matrix: row length uniform in [lmin, lmax]; each column
    with probability p_band at a uniform offset in [-band, band] from the
    diagonal, otherwise uniform in [0, N); values uniform in (-1, 1)."""
    rows = np.arange(N, dtype=np.int64)
    rowlen = rng.randint(rng.stream_key(seed, _T_ROWLEN), rows, lmin, lmax)

    def draw(ent, own, attempt):
        kind = rng.uniform01(rng.stream_key(seed, _T_KIND, attempt), ent) < p_band
        off = rng.randint(rng.stream_key(seed, _T_BAND, attempt), ent, -band, band)
        uni = rng.randint(rng.stream_key(seed, _T_UNI, attempt), ent, 0, N - 1)
        return np.where(kind, own + off, uni)

    rowptr, col = _random_pattern(N, N, rowlen, draw, lmax)
    val = rng.uniform(rng.stream_key(seed, _T_VAL), np.arange(rowptr[-1]), -1.0, 1.0)
    return _finish(N, N, rowptr, col, val, kind="irregular_band", lmin=lmin, lmax=lmax, band=band,
                   p_band=p_band, seed=seed)


def powerlaw_lengths(N: int, kmin: int, kmax: int, exponent: float, key) -> np.ndarray:
    """Row lengths k in [kmin, kmax] with P(k) proportional to k**-exponent,
    sampled by inverting the discrete CDF."""
    ks = np.arange(kmin, kmax + 1, dtype=np.float64)
    pmf = ks ** (-exponent)
    cdf = np.cumsum(pmf) / pmf.sum()
    u = rng.uniform01(key, np.arange(N))
    pos = np.searchsorted(cdf, u, side="right")
    return (kmin + np.minimum(pos, kmax - kmin)).astype(np.int64)


def powerlaw(N: int = 1 << 20, kmin: int = 1, kmax: int = 256, exponent: float = 2.0,
             seed: int = BASE_SEED + 3, fp32_values: bool = True) -> CSR:
    """Power-law row lengths, uniform random distinct columns, N(0,1) values
    (rounded to float32 when ``fp32_values``; still returned as float64)."""
    rowlen = powerlaw_lengths(N, kmin, kmax, exponent, rng.stream_key(seed, _T_ROWLEN))

    def draw(ent, own, attempt):
        return rng.randint(rng.stream_key(seed, _T_UNI, attempt), ent, 0, N - 1)

    rowptr, col = _random_pattern(N, N, rowlen, draw, kmax)
    val = rng.normal(rng.stream_key(seed, _T_VAL), np.arange(rowptr[-1]))
    if fp32_values:
        val = val.astype(np.float32).astype(np.float64)
    return _finish(N, N, rowptr, col, val, kind="powerlaw", kmin=kmin, kmax=kmax,
                   exponent=exponent, seed=seed)


# --------------------------------------------------------------------------- vectors

def block_vector(nrows: int, w: int, seed: int, tag: int = _T_X, lo: float = -1.0, hi: float = 1.0):
    """Row-major nrows x w block vector, uniform in [lo, hi)."""
    ctr = np.arange(nrows * w, dtype=np.int64)
    return rng.uniform(rng.stream_key(seed, tag), ctr, lo, hi).reshape(nrows, w)


def normal_block(nrows: int, w: int, seed: int, tag: int = _T_X):
    ctr = np.arange(nrows * w, dtype=np.int64)
    return rng.normal(rng.stream_key(seed, tag), ctr).reshape(nrows, w)


def laplace3d_mode(n: int, p: int, q: int, r: int) -> np.ndarray:
    """Sine mode sin(p*pi*(i+1)/(n+1)) sin(q*pi*(j+1)/(n+1)) sin(r*pi*(k+1)/(n+1))
    of the Dirichlet grid, in the row order of :func:`laplace3d`."""
    t = np.arange(1, n + 1) * np.pi / (n + 1)
    si, sj, sk = np.sin(p * t), np.sin(q * t), np.sin(r * t)
    return (sk[:, None, None] * sj[None, :, None] * si[None, None, :]).ravel()


def laplace2d_mode(s: int, p: int, q: int) -> np.ndarray:
    """Sine mode sin(p*pi*(i+1)/(s+1)) sin(q*pi*(j+1)/(s+1)), row order of :func:`laplace2d`."""
    t = np.arange(1, s + 1) * np.pi / (s + 1)
    return (np.sin(q * t)[:, None] * np.sin(p * t)[None, :]).ravel()


def lattice_plane_wave(n: int, p: int, q: int, r: int) -> np.ndarray:
    """cos(2 pi (p i + q j + r k)/n) on the periodic n^3 lattice of :func:`anderson3d`."""
    t = 2.0 * np.pi * np.arange(n) / n
    ph = (r * t)[:, None, None] + (q * t)[None, :, None] + (p * t)[None, None, :]
    return np.cos(ph).ravel()


# --------------------------------------------------------------------------- the five workloads

def workload_laplace(n: int = 32, seed: int = BASE_SEED + 0):
    """3D 7-point Dirichlet Laplacian and one uniform(-1,1) vector."""
    A = laplace3d(n)
    x = block_vector(A.nrows, 1, seed + 1)
    return A, x


def workload_irregular(N: int = 1 << 21, seed: int = BASE_SEED + 1, **kw):
    """Irregular band matrix with x, y0, z0 for the augmented product."""
    A = irregular_band(N, seed=seed, **kw)
    x = block_vector(N, 1, seed, _T_X)
    y0 = block_vector(N, 1, seed, _T_X + 100)
    z0 = block_vector(N, 1, seed, _T_X + 200)
    return A, x, y0, z0


def workload_anderson(n: int = 128, w: int = 16, seed: int = BASE_SEED + 2, disorder: bool = True):
    A = anderson3d(n, seed=seed, disorder=disorder)
    x = block_vector(A.nrows, w, seed, _T_X)
    return A, x


def workload_powerlaw(N: int = 1 << 20, w: int = 4, seed: int = BASE_SEED + 3, **kw):
    """Power-law matrix with float32-representable x and upstream gradient g."""
    A = powerlaw(N, seed=seed, **kw)
    x = normal_block(N, w, seed, _T_X).astype(np.float32).astype(np.float64)
    g = normal_block(N, w, seed, _T_X + 100).astype(np.float32).astype(np.float64)
    return A, x, g


def cg_batch_specs(count: int = 64, smin: int = 64, smax: int = 512, wmin: int = 1, wmax: int = 8,
                   seed: int = BASE_SEED + 4):
    """Grid sides and right-hand-side widths of a batch of 2D Laplacian systems."""
    m = np.arange(count)
    sides = rng.randint(rng.stream_key(seed, _T_SIZE), m, smin, smax)
    widths = rng.randint(rng.stream_key(seed, _T_W), m, wmin, wmax)
    return [(int(s), int(w)) for s, w in zip(sides, widths)]


def workload_cg_batch(count: int = 64, smin: int = 64, smax: int = 512, wmin: int = 1, wmax: int = 8,
                      seed: int = BASE_SEED + 4, shift: float = 0.01):
    """Batch of (A_m, B_m): A_m = L_2D(s_m) + shift*I and a uniform(-1,1) right-hand
    side block of width w_m."""
    out = []
    for m, (s, w) in enumerate(cg_batch_specs(count, smin, smax, wmin, wmax, seed)):
        A = laplace2d(s, shift)
        B = block_vector(A.nrows, w, seed, _T_RHS * 1000 + m)
        out.append((A, B))
    return out
