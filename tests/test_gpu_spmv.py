"""GPU parity of the augmented SpMMV (through the C ABI) against the oracle.

Covers every subset of the augmentation flags, block widths 1..33 (padded
power-of-two variants, the masked generic path and the 32-column tiling),
chunk heights and sort windows, all five precision pairs, row- and
column-major block vectors with padded leading dimensions, rectangular
matrices and the degenerate shapes (empty matrix, empty rows, one row, fewer
rows than C, a row far longer than the rest)."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import assert_close, dot_bound, run_case, to_dev
from tests.test_oracle_format import random_csr
from workloads import generators as gen
from workloads.generators import CSR

pytestmark = pytest.mark.gpu

FLAGS = ["scale", "shift", "vshift", "axpby", "dot_yy", "dot_xy", "dot_xx", "chain"]


def flag_sets():
    for bits in range(1 << len(FLAGS)):
        f = {n for k, n in enumerate(FLAGS) if bits >> k & 1}
        if "shift" in f and "vshift" in f:
            continue
        yield f


ALL = {"scale", "vshift", "axpby", "dot_yy", "dot_xy", "dot_xx", "chain"}


@pytest.fixture(scope="module")
def irregular():
    return gen.irregular_band(3001, lmin=0, lmax=40, band=200, seed=12)


@pytest.mark.parametrize("w", [1, 3, 16])
def test_all_flag_subsets(cuda_ok, irregular, w):
    mat = sellcs.SellMatrix(irregular, C=32, sigma=256)
    for f in flag_sets():
        run_case(irregular, 32, 256, w, f, mat=mat, seed=len(f))


@pytest.mark.parametrize("C,sigma", list(itertools.product([8, 16, 32], [1, 32, 256, 1024])))
def test_chunk_and_window_grid(cuda_ok, irregular, C, sigma):
    mat = sellcs.SellMatrix(irregular, C=C, sigma=sigma)
    for w in (1, 2, 3, 4, 7, 8, 16, 33):
        run_case(irregular, C, sigma, w, ALL, mat=mat, seed=w)
    run_case(irregular, C, sigma, 1, set(), mat=mat)


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f64"), ("bf16", "f64"), ("f32", "f32"),
                                     ("bf16", "f32")])
@pytest.mark.parametrize("w", [1, 2, 4, 5, 8, 16, 32])
def test_precisions(cuda_ok, irregular, vdt, xdt, w):
    run_case(irregular, 32, 256, w, ALL, vdt=vdt, xdt=xdt, seed=w)


@pytest.mark.parametrize("w", [1, 2, 4, 6, 16])
@pytest.mark.parametrize("layout,pad", [("row", 3), ("col", 0), ("col", 5)])
def test_layouts_and_leading_dimension(cuda_ok, irregular, w, layout, pad):
    run_case(irregular, 32, 32, w, ALL, layout=layout, ld_pad=pad, seed=w)


def test_rectangular(cuda_ok):
    rng = np.random.default_rng(4)
    A = random_csr(300, 517, 0.05, rng)
    for w in (1, 4, 9):
        run_case(A, 16, 64, w, {"scale", "axpby", "chain", "dot_yy"}, seed=w)
    # more columns than rows: the shift and the x-dots use x's first nrows
    # rows (a process's rows with its halo columns appended)
    run_case(A, 16, 64, 2, {"scale", "shift", "dot_xy", "dot_xx", "dot_yy"}, seed=11)
    run_case(A, 32, 1, 3, {"vshift", "axpby", "dot_xy"}, seed=12)
    B = random_csr(517, 300, 0.05, rng)
    with pytest.raises(sellcs.SpError) as e:
        run_case(B, 16, 64, 2, {"dot_xy"})
    assert e.value.code == sellcs.SP_ERR_DIM


@pytest.mark.parametrize("N", [1, 5, 31, 33, 64])
def test_small_shapes(cuda_ok, N):
    rng = np.random.default_rng(N)
    A = random_csr(N, N, 0.4, rng)
    for C, sigma in [(1, 1), (4, 3), (32, 1), (32, 1000), (64, 64)]:
        run_case(A, C, sigma, 1, ALL, seed=C)
        run_case(A, C, sigma, 5, ALL, seed=C + 1)


def test_empty_rows_and_long_row(cuda_ok):
    N = 2000
    rng = np.random.default_rng(8)
    lens = rng.integers(0, 4, N)
    lens[rng.integers(N)] = N  # one dense row
    lens[::7] = 0
    rowptr = np.zeros(N + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    col = np.concatenate([np.sort(rng.choice(N, size=l, replace=False)) for l in lens]).astype(np.int32)
    A = gen.CSR(N, N, rowptr, col, rng.uniform(-1, 1, rowptr[-1]))
    for sigma in (1, 128, N):
        run_case(A, 32, sigma, 1, ALL)
        run_case(A, 32, sigma, 8, ALL)


def test_empty_matrix(cuda_ok):
    A = gen.CSR(0, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    mat = sellcs.SellMatrix(A, C=32, sigma=1)
    assert mat.info()["nchunks"] == 0
    x = torch.zeros(0, 2, dtype=torch.float64, device="cuda")
    y = torch.zeros(0, 2, dtype=torch.float64, device="cuda")
    dot = torch.full((6,), 7.0, dtype=torch.float64, device="cuda")
    sellcs.spmv(mat, x, y, dot_yy=True, dot_xx=True, dot=dot)
    d = dot.cpu().numpy()
    assert d[0] == 0 and d[1] == 0 and d[4] == 0 and d[5] == 0 and d[2] == 7.0


def test_all_zero_pattern(cuda_ok):
    N = 100
    A = gen.CSR(N, N, np.zeros(N + 1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    run_case(A, 32, 1, 3, ALL)


def test_beta_off_ignores_nan_y_and_deterministic_dots(cuda_ok):
    A = gen.irregular_band(20000, band=500, seed=3)
    mat = sellcs.SellMatrix(A, C=32, sigma=256)
    x = to_dev(gen.block_vector(A.nrows, 4, 1))
    outs = []
    for _ in range(3):
        y = torch.full((A.nrows, 4), float("nan"), dtype=torch.float64, device="cuda")
        d = sellcs.spmv(mat, x, y, dot_yy=True, dot_xy=True)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        outs.append(d.cpu().numpy().copy())
    np.testing.assert_array_equal(outs[0][:8], outs[1][:8])
    np.testing.assert_array_equal(outs[0][:8], outs[2][:8])


def test_aliasing_and_argument_errors(cuda_ok, irregular):
    mat = sellcs.SellMatrix(irregular, C=32, sigma=1)
    x = to_dev(np.ones((irregular.nrows, 2)))
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv(mat, x, x)
    assert e.value.code == sellcs.SP_ERR_ARG
    y = torch.zeros_like(x)
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv(mat, x, y, z=x, delta=1.0, eta=1.0)
    assert e.value.code == sellcs.SP_ERR_ARG
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv(mat, x[:-1], y)
    assert e.value.code == sellcs.SP_ERR_DIM
    with pytest.raises(sellcs.SpError) as e:
        sellcs.spmv(mat, x.float(), y.float())  # f64 values need f64 vectors
    assert e.value.code == sellcs.SP_ERR_DTYPE


def test_dot_to_host_pointer(cuda_ok, irregular):
    import ctypes as ct
    mat = sellcs.SellMatrix(irregular, C=32, sigma=32)
    X = gen.block_vector(irregular.nrows, 3, 9)
    x = to_dev(X)
    y = torch.zeros_like(x)
    hx, hy = sellcs.sp_dense_view(x), sellcs.sp_dense_view(y)
    host = np.full(9, np.nan)
    o, keep = sellcs.make_opts(3, dot_xx=True, dot_yy=True, dot_ptr=host.ctypes.data_as(ct.c_void_p),
                               dot_host=True)
    sellcs.check(sellcs.lib().sp_spmv(hy, mat.handle, hx, ct.byref(o), sellcs._stream(None)), "spmv")
    yr, dr, _ = oracle.spmmv(irregular, X, dot_yy=True, dot_xx=True)
    e = 1e-12 * oracle.spmmv_scale(irregular, X)
    N = irregular.nrows
    assert_close(host[6:], dr[6:], dot_bound("dot_xx", yr, X, e, "f64", N), 1.0, "host dot_xx")
    assert_close(host[:3], dr[:3], dot_bound("dot_yy", yr, X, e, "f64", N), 1.0, "host dot_yy")
    assert np.all(np.isnan(host[3:6]))
    sellcs.sp_dense_destroy(hx)
    sellcs.sp_dense_destroy(hy)


@pytest.mark.parametrize("C", [1, 2, 4, 8, 16])
def test_threads_per_row_long_rows(cuda_ok, C):
    """Small C gives each row T = 32 / (C * lanes per row) lanes (long power-law rows)."""
    A = gen.powerlaw(6000, seed=14)
    mat = sellcs.SellMatrix(A, C=C, sigma=6000)
    for w in (1, 2, 3, 4, 8):
        run_case(A, C, 6000, w, ALL, mat=mat, seed=w)
    for vdt, xdt in (("f32", "f32"), ("bf16", "f32")):
        run_case(A, C, 64, 4, ALL, vdt=vdt, xdt=xdt)


@pytest.fixture(scope="module")
def irregular_large():
    """About 400k rows (more 32-row blocks than warps in one grid, so the moving
    front takes several rounds), empty rows included."""
    return gen.irregular_band(400_003, lmin=0, lmax=24, band=2000, seed=31)


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f32")])
@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 256), (8, 1 << 20)])
@pytest.mark.parametrize("w", [1, 16])
def test_work_order_does_not_change_results(cuda_ok, irregular_large, vdt, xdt, C, sigma, w):
    """Moving front, contiguous ranges and the automatic choice (and with them
    the lockstep or per-lane row loop, chosen by the row-length spread) give
    bit-identical y; each matches the oracle."""
    A = irregular_large
    ys = []
    for order in ("auto", "front", "ranges"):
        m = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=vdt, order=order)
        y, _, _ = run_case(A, C, sigma, w, {"scale", "shift", "axpby", "dot_yy", "dot_xy", "chain"}, vdt=vdt,
                           xdt=xdt, mat=m, seed=7)
        m.close()
        ys.append(y)
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f32"), ("bf16", "f64")])
@pytest.mark.parametrize("w", [8, 16, 32])
def test_dynamic_order_repeats_and_matches_static(cuda_ok, irregular_large, vdt, xdt, w):
    """Products on wide row-major blocks without fused reductions take their
    rows in dynamic order (warps draw runs of slots from a counter that the
    last warp resets).  Three calls in a row give the same bits, the same bits
    as the product with dot products (static order), and match the oracle."""
    A = irregular_large
    m = sellcs.SellMatrix(A, C=32, sigma=256, dtype=vdt)
    plain = {"scale", "shift", "axpby", "chain"}
    ys = [run_case(A, 32, 256, w, plain, vdt=vdt, xdt=xdt, mat=m, seed=11)[0] for _ in range(3)]
    y_static = run_case(A, 32, 256, w, plain | {"dot_yy"}, vdt=vdt, xdt=xdt, mat=m, seed=11)[0]
    m.close()
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
    assert np.array_equal(ys[0], y_static)


def test_float64_extreme_magnitudes(cuda_ok):
    """x entries and matrix values of extreme magnitude (1e60, 3e-30, 1e45
    scaling), exact zeros and an infinity: the float64 tolerance holds and a
    non-finite x entry reaches exactly the rows that use it."""
    rng = np.random.default_rng(21)
    A = random_csr(3000, 3000, 0.01, rng)
    # x with entries far outside [2^-40, 2^40], exact zeros and a few infinities
    X = rng.uniform(-1, 1, (3000, 3))
    X[::97, 0] = 1e60
    X[::89, 1] = 3e-30
    X[::83, 2] = 0.0
    run_case(A, 32, 64, 3, {"scale", "axpby", "dot_xx"}, seed=1)  # in-range baseline
    import oracle as orc
    for vals in (A.val, A.val * 1e45):
        B = gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, vals)
        m = sellcs.SellMatrix(B, C=32, sigma=64)
        x = to_dev(X)
        y = torch.zeros_like(x)
        sellcs.spmv(m, x, y)
        torch.cuda.synchronize()
        yr = orc.spmmv(B, X)[0]
        s = orc.spmmv_scale(B, X)
        assert np.all(np.abs(y.cpu().numpy() - yr) <= 1e-12 * s + 1e-300)
    X[5, 0] = np.inf
    m = sellcs.SellMatrix(A, C=32, sigma=64)
    y = torch.zeros(3000, 3, dtype=torch.float64, device="cuda")
    sellcs.spmv(m, to_dev(X), y)
    yr = orc.spmmv(A, X)[0]
    yg = y.cpu().numpy()
    # a non-finite x entry reaches exactly the rows that use it (the oracle's
    # compensated sum turns inf into nan, so compare finiteness only)
    np.testing.assert_array_equal(np.isfinite(yg), np.isfinite(yr))
    fin = np.isfinite(yr)
    s = orc.spmmv_scale(A, np.where(np.isfinite(X), X, 0.0))
    assert np.all(np.abs(yg[fin] - yr[fin]) <= 1e-12 * s[fin] + 1e-300)


@pytest.mark.parametrize("C,sigma", [(32, 1), (32, 32), (32, 256), (64, 64), (64, 1)])
def test_lockstep_rows_exact_tail(cuda_ok, C, sigma):
    """Single float64 vectors with widely spread row lengths take the lockstep
    row loop, whose last steps stop at the chunk's longest row (a jump into
    the unrolled sequence).  Rows of every length from 0 to 90 (every tail
    length), padding rows in the last chunk (N = 32 k + 5): y, z and the dots
    against the oracle, for every work order, bit-identical between the
    orders."""
    rng = np.random.default_rng(C + sigma)
    N = 32 * 97 + 5
    lens = rng.integers(0, 91, N)
    lens[rng.random(N) < 0.1] = 0
    rowptr = np.zeros(N + 1, np.int64)
    rowptr[1:] = np.cumsum(lens)
    col = np.concatenate([np.sort(rng.choice(N, int(k), replace=False)) for k in lens]).astype(np.int32)
    A = CSR(N, N, rowptr, col, rng.uniform(-1, 1, int(rowptr[-1])))
    ys = []
    for order in ("auto", "front", "ranges"):
        m = sellcs.SellMatrix(A, C=C, sigma=sigma, order=order)
        y, _, _ = run_case(A, C, sigma, 1, {"scale", "shift", "axpby", "dot_yy", "dot_xy", "chain"}, mat=m, seed=3)
        run_case(A, C, sigma, 1, set(), mat=m, seed=4)
        run_case(A, C, sigma, 1, {"scale", "axpby"}, mat=m, seed=5)
        m.close()
        ys.append(y)
    assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])
