"""Pins of the oracle's SELL-C-sigma construction (CPU only).

What fixes the answer here, independently of the oracle's own code:
* a hand-worked example of the format definition (tests/golden);
* the paper's format identities: SELL-1-1 is CRS/CSR, SELL-n-1 is
  ITPACK/ELLPACK, SELL-C-1 is Sliced ELLPACK (Sec. "Sparse matrix storage");
* the permutation against Python's stable ``sorted`` per window;
* brute force over many tiny random matrices: exact CSR -> SELL -> CSR round
  trips and the layout invariants.
"""
import itertools

import numpy as np
import pytest

import oracle
from tests.conftest import read_golden
from workloads.generators import CSR, irregular_band, laplace3d, powerlaw


def _csr_from_golden(g):
    rowptr = g["rowptr"].astype(np.int64)
    return CSR(int(g["nrows"][0]), int(g["nrows"][0]), rowptr, g["col"].astype(np.int32), g["val"])


def random_csr(N, ncols, density, rng, empty_rows=True):
    rows = []
    for i in range(N):
        m = rng.random(ncols) < density
        if not empty_rows and not m.any():
            m[rng.integers(ncols)] = True
        rows.append(np.nonzero(m)[0])
    rowptr = np.zeros(N + 1, np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32) if rowptr[-1] else np.zeros(0, np.int32)
    val = rng.uniform(-1, 1, int(rowptr[-1]))
    return CSR(N, ncols, rowptr, col, val)


def test_golden_example():
    g = read_golden("sell_5x5_c2_s4.txt")
    A = _csr_from_golden(g)
    S = oracle.sell_from_csr(A, int(g["C"][0]), int(g["sigma"][0]))
    for k in ("perm", "slotlen", "chunklen", "chunkptr"):
        np.testing.assert_array_equal(getattr(S, k), g[k].astype(np.int64), err_msg=k)
    np.testing.assert_array_equal(S.col, g["col_sell"].astype(np.int32))
    np.testing.assert_array_equal(S.val, g["val_sell"])
    y, _, _ = oracle.spmmv(A, g["x"])
    np.testing.assert_array_equal(y[:, 0], g["y"])


def test_sell_1_1_is_csr():
    A = irregular_band(500, lmin=0, lmax=9, band=20, seed=7)
    S = oracle.sell_from_csr(A, 1, 1)
    np.testing.assert_array_equal(S.perm, np.arange(A.nrows))
    np.testing.assert_array_equal(S.chunkptr, A.rowptr)
    np.testing.assert_array_equal(S.chunklen, np.diff(A.rowptr))
    np.testing.assert_array_equal(S.col, A.col)
    np.testing.assert_array_equal(S.val, A.val)


def _ellpack(A, rows):
    """ELLPACK of the given rows: width = longest row, column-major, zero pad."""
    L = max([int(A.rowptr[i + 1] - A.rowptr[i]) for i in rows] + [0])
    val = np.zeros((L, len(rows)))
    col = np.zeros((L, len(rows)), np.int64)
    for r, i in enumerate(rows):
        seg = slice(A.rowptr[i], A.rowptr[i + 1])
        n = A.rowptr[i + 1] - A.rowptr[i]
        val[:n, r] = A.val[seg]
        col[:n, r] = A.col[seg]
        col[n:, r] = A.col[A.rowptr[i + 1] - 1] if n else 0
    return L, val.ravel(), col.ravel()


def test_sell_n_1_is_ellpack():
    A = irregular_band(300, lmin=1, lmax=12, band=30, seed=3)
    S = oracle.sell_from_csr(A, A.nrows, 1)
    L, v, c = _ellpack(A, range(A.nrows))
    assert S.nchunks == 1 and S.chunklen[0] == L
    np.testing.assert_array_equal(S.val, v)
    np.testing.assert_array_equal(S.col, c)


@pytest.mark.parametrize("C", [2, 4, 8, 32])
def test_sell_c_1_is_sliced_ellpack(C):
    A = irregular_band(203, lmin=0, lmax=15, band=25, seed=11)
    S = oracle.sell_from_csr(A, C, 1)
    parts_v, parts_c = [], []
    for c0 in range(0, A.nrows, C):
        rows = list(range(c0, min(c0 + C, A.nrows)))
        L, v, cc = _ellpack(A, rows)
        # the last slice is padded with empty rows up to C
        vv = np.zeros((L, C))
        ccc = np.zeros((L, C), np.int64)
        vv[:, :len(rows)] = v.reshape(L, len(rows))
        ccc[:, :len(rows)] = cc.reshape(L, len(rows))
        parts_v.append(vv.ravel())
        parts_c.append(ccc.ravel())
    np.testing.assert_array_equal(S.val, np.concatenate(parts_v))
    np.testing.assert_array_equal(S.col, np.concatenate(parts_c))


def _check_invariants(A, S):
    N, C, sigma = A.nrows, S.C, S.sigma
    lens = np.diff(A.rowptr)
    nch = (N + C - 1) // C
    assert S.perm.size == nch * C
    assert sorted(S.perm[:N].tolist()) == list(range(N))
    assert np.all(S.perm[N:] == -1) and np.all(S.slotlen[N:] == 0)
    # permutation = stable descending sort of each window (Python's sort is stable)
    for w0 in range(0, N, sigma):
        w1 = min(w0 + sigma, N)
        ref = sorted(range(w0, w1), key=lambda i: -lens[i])
        assert S.perm[w0:w1].tolist() == ref
    np.testing.assert_array_equal(S.slotlen[:N], lens[S.perm[:N]])
    assert int(S.slotlen.sum()) == A.nnz
    for c in range(nch):
        assert S.chunklen[c] == S.slotlen[c * C:(c + 1) * C].max(initial=0)
        assert S.chunkptr[c + 1] - S.chunkptr[c] == C * S.chunklen[c]
        for r in range(C):
            s = c * C + r
            j = np.arange(S.slotlen[s], S.chunklen[c])
            assert np.all(S.val[S.chunkptr[c] + j * C + r] == 0.0)


def test_bruteforce_tiny_roundtrip():
    rng = np.random.default_rng(5)
    count = 0
    for N in range(1, 7):
        for trial in range(12):
            A = random_csr(N, N, rng.uniform(0.1, 0.9), rng)
            for C, sigma in itertools.product([1, 2, 4, 8, 32], [1, 2, 4, N]):
                S = oracle.sell_from_csr(A, C, sigma)
                _check_invariants(A, S)
                rp, col, val = oracle.sell_to_csr(S)
                np.testing.assert_array_equal(rp, A.rowptr)
                np.testing.assert_array_equal(col, A.col)
                np.testing.assert_array_equal(val, A.val)
                count += 1
    assert count == 6 * 12 * 20


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 256), (8, 32), (16, 1024), (32, 100_000)])
def test_roundtrip_workloads(C, sigma):
    for A in (laplace3d(8), irregular_band(3000, band=100, seed=2), powerlaw(3000, seed=4)):
        S = oracle.sell_from_csr(A, C, sigma)
        _check_invariants(A, S)
        rp, col, val = oracle.sell_to_csr(S)
        np.testing.assert_array_equal(rp, A.rowptr)
        np.testing.assert_array_equal(col, A.col)
        np.testing.assert_array_equal(val, A.val)


def test_sigma_cuts_padding():
    """Sorting inside windows can only lower the stored-entry count (the reason
    for sigma in the paper); with sigma = N the padding is minimal."""
    A = powerlaw(4096, seed=9)
    stored = [oracle.sell_from_csr(A, 32, s).nstored for s in (1, 32, 256, 4096)]
    assert all(a >= b for a, b in zip(stored, stored[1:]))
    assert stored[-1] < stored[0]
