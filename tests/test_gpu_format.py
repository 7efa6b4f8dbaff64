"""GPU construction of SELL-C-sigma against the oracle, bit for bit:
permutation, per-slot lengths, chunk lengths and offsets, column indices,
padding and values (including their float32 / bfloat16 rounding), the
transposed matrix, the CSR round trip, value-only updates and value clones."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.conftest import read_golden
from tests.test_oracle_format import random_csr
from workloads import generators as gen

pytestmark = pytest.mark.gpu


def assert_same_sell(exp, ref, vdt="f64"):
    np.testing.assert_array_equal(exp["perm"], ref.perm)
    np.testing.assert_array_equal(exp["slotlen"], ref.slotlen)
    np.testing.assert_array_equal(exp["chunklen"], ref.chunklen)
    np.testing.assert_array_equal(exp["chunkptr"], ref.chunkptr)
    np.testing.assert_array_equal(exp["col"], ref.col)
    np.testing.assert_array_equal(exp["val"], oracle.round_values(ref.val, vdt))


def transpose_csr(A):
    """CSR of A^T: entries ordered by (column, row), by a stable argsort."""
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    order = np.argsort(A.col, kind="stable")
    rp = np.zeros(A.ncols + 1, np.int64)
    np.add.at(rp, A.col.astype(np.int64) + 1, 1)
    rp = np.cumsum(rp)
    return gen.CSR(A.ncols, A.nrows, rp, rows[order].astype(np.int32), A.val[order])


def test_golden(cuda_ok):
    g = read_golden("sell_5x5_c2_s4.txt")
    A = gen.CSR(5, 5, g["rowptr"].astype(np.int64), g["col"].astype(np.int32), g["val"])
    m = sellcs.SellMatrix(A, C=2, sigma=4)
    e = m.export_sell()
    for k in ("perm", "slotlen", "chunklen", "chunkptr"):
        np.testing.assert_array_equal(e[k], g[k].astype(np.int64), err_msg=k)
    np.testing.assert_array_equal(e["col"], g["col_sell"])
    np.testing.assert_array_equal(e["val"], g["val_sell"])


def test_tiny_bruteforce(cuda_ok):
    rng = np.random.default_rng(0)
    for N in range(1, 7):
        for t in range(4):
            A = random_csr(N, N, rng.uniform(0.1, 0.9), rng)
            for C, sigma in itertools.product([1, 2, 4, 8, 32], [1, 2, 4, N]):
                m = sellcs.SellMatrix(A, C=C, sigma=sigma)
                assert_same_sell(m.export_sell(), oracle.sell_from_csr(A, C, sigma))
                rp, col, val = m.to_csr()
                np.testing.assert_array_equal(rp, A.rowptr)
                np.testing.assert_array_equal(col, A.col)
                np.testing.assert_array_equal(val, A.val)


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 256), (8, 32), (16, 1024), (32, 1 << 30), (7, 100)])
@pytest.mark.parametrize("vdt", ["f64", "f32", "bf16"])
def test_workload_patterns(cuda_ok, C, sigma, vdt):
    for A in (gen.laplace3d(10), gen.irregular_band(20000, band=300, seed=2), gen.powerlaw(20000, seed=4)):
        m = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=vdt)
        assert_same_sell(m.export_sell(), oracle.sell_from_csr(A, C, sigma), vdt)
        inf = m.info()
        assert inf["nnz"] == A.nnz and inf["maxrowlen"] == np.diff(A.rowptr).max()


def test_transpose_pattern(cuda_ok):
    for A in (gen.powerlaw(5000, seed=6), random_csr(300, 700, 0.02, np.random.default_rng(2))):
        for C, sigma in [(32, 1), (32, 256), (8, 64)]:
            m = sellcs.SellMatrix(A, C=C, sigma=sigma, with_transpose=True)
            assert_same_sell(m.export_sell(transpose=True), oracle.sell_from_csr(transpose_csr(A), C, sigma))


def test_update_values_and_clone(cuda_ok):
    A = gen.powerlaw(8000, seed=7)
    m = sellcs.SellMatrix(A, C=32, sigma=128, with_transpose=True)
    new = gen.normal_block(A.nnz, 1, 33)[:, 0]
    B = gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, new)
    m.update_values(new)  # host input
    assert_same_sell(m.export_sell(), oracle.sell_from_csr(B, 32, 128))
    assert_same_sell(m.export_sell(transpose=True), oracle.sell_from_csr(transpose_csr(B), 32, 128))
    new2 = new * 0.5 - 1.0
    m.update_values(torch.from_numpy(new2).cuda())  # device input
    B2 = gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, new2)
    assert_same_sell(m.export_sell(), oracle.sell_from_csr(B2, 32, 128))
    m.update_values(torch.from_numpy(new2.astype(np.float32)).cuda())  # float32 device input
    assert_same_sell(m.export_sell(), oracle.sell_from_csr(
        gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, new2.astype(np.float32).astype(np.float64)), 32, 128))
    for dt in ("f32", "bf16"):
        c = m.clone(dt)
        assert_same_sell(c.export_sell(), oracle.sell_from_csr(
            gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, new2.astype(np.float32).astype(np.float64)), 32, 128), dt)


def test_malformed_csr_rejected(cuda_ok):
    rp = np.array([0, 2, 1, 3], np.int64)  # decreasing
    A = gen.CSR(3, 3, rp, np.array([0, 1, 2], np.int32), np.ones(3))
    with pytest.raises(sellcs.SpError) as e:
        sellcs.SellMatrix(A)
    assert e.value.code == sellcs.SP_ERR_FORMAT
    A = gen.CSR(2, 2, np.array([0, 1, 2], np.int64), np.array([0, 5], np.int32), np.ones(2))
    with pytest.raises(sellcs.SpError) as e:
        sellcs.SellMatrix(A)
    assert e.value.code == sellcs.SP_ERR_FORMAT


def test_device_csr_input(cuda_ok):
    A = gen.irregular_band(5000, band=100, seed=5)
    t = (A.nrows, A.ncols, torch.from_numpy(A.rowptr).cuda(), torch.from_numpy(A.col).cuda(),
         torch.from_numpy(A.val).cuda())
    m = sellcs.SellMatrix(t, C=32, sigma=64)
    assert_same_sell(m.export_sell(), oracle.sell_from_csr(A, 32, 64))
