"""GPU adjoint of y = A x against the oracle's gradient, float64 central finite
differences and torch.autograd.gradcheck; the power-law workload at full size
(N = 2^20, block width 4, float32)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import autograd, sellcs
from tests.gpu_helpers import U32, assert_close, to_dev
from tests.test_oracle_format import random_csr
from tests.test_oracle_grad_cg import _slice
from workloads import generators as gen

pytestmark = pytest.mark.gpu


def _abs(A):
    return gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, np.abs(A.val))


def check_adjoint(A, w, C, sigma, xdt, seed=0):
    rng = np.random.default_rng(seed)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    vdt = xdt
    X = rng.normal(size=(A.ncols, w))
    G = rng.normal(size=(A.nrows, w))
    vals = A.val
    if xdt == "f32":
        X, G = X.astype(np.float32).astype(np.float64), G.astype(np.float32).astype(np.float64)
        vals = oracle.round_values(A.val, "f32")
    Ar = gen.CSR(A.nrows, A.ncols, A.rowptr, A.col, vals)
    m = sellcs.SellMatrix(Ar, C=C, sigma=sigma, dtype=vdt, with_transpose=True)
    x, g = to_dev(X, tdt), to_dev(G, tdt)
    dx = torch.full((A.ncols, w), float("nan"), dtype=tdt, device="cuda")
    dv = torch.full((A.nnz,), float("nan"), dtype=tdt, device="cuda")
    sellcs.spmv_adjoint(m, g, x=x, dx=dx, dvals=dv)
    torch.cuda.synchronize()
    ref_dx = oracle.spmmv_transpose(Ar, G)
    ref_dv = oracle.sampled_product(Ar, G, X)
    collen = np.bincount(A.col, minlength=A.ncols)
    if xdt == "f64":
        tdx, tdv = 1e-12, 1e-12
    else:
        tdx = 1.1 * (collen.max(initial=0) + 6) * U32
        tdv = 1.1 * (w + 6) * U32
    s_dx = oracle.spmmv_transpose(_abs(Ar), np.abs(G)) + (np.abs(ref_dx) if xdt == "f32" else 0)
    s_dv = oracle.sampled_product(A, np.abs(G), np.abs(X)) + (np.abs(ref_dv) if xdt == "f32" else 0)
    assert_close(dx.double().cpu().numpy(), ref_dx, s_dx, tdx, f"dx w={w} C={C} s={sigma} {xdt}")
    assert_close(dv.double().cpu().numpy(), ref_dv, s_dv, tdv, f"dvals w={w} C={C} s={sigma} {xdt}")


@pytest.mark.parametrize("xdt", ["f64", "f32"])
@pytest.mark.parametrize("w", [1, 2, 3, 4, 8, 16, 32])
def test_adjoint_random(cuda_ok, xdt, w):
    rng = np.random.default_rng(w)
    A = random_csr(700, 700, 0.01, rng)
    for C, sigma in [(32, 1), (8, 64), (32, 700)]:
        check_adjoint(A, w, C, sigma, xdt, seed=C)


def test_adjoint_rectangular(cuda_ok):
    A = random_csr(300, 1000, 0.02, np.random.default_rng(3))
    check_adjoint(A, 4, 16, 32, "f64")


def test_gradcheck_small(cuda_ok):
    A = random_csr(40, 40, 0.15, np.random.default_rng(11))
    m = sellcs.SellMatrix(A, C=8, sigma=16, with_transpose=True)
    vals = torch.tensor(A.val, dtype=torch.float64, device="cuda", requires_grad=True)
    x = torch.randn(40, 3, dtype=torch.float64, device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda v, xx: autograd.spmv(m, v, xx), (vals, x), eps=1e-6, atol=1e-8)


def test_finite_differences_powerlaw_slice(cuda_ok):
    """FP64 central differences (h = 1e-6) of L = sum(g * A x) on a 4096-row
    slice of the power-law matrix against the GPU gradient."""
    full = gen.powerlaw(1 << 14, seed=gen.BASE_SEED + 3)
    A = _slice(full, 4096)
    w = 4
    X = gen.normal_block(A.nrows, w, 1)
    G = gen.normal_block(A.nrows, w, 2)
    m = sellcs.SellMatrix(A, C=32, sigma=256, with_transpose=True)
    vals = torch.tensor(A.val, device="cuda", requires_grad=True)
    x = to_dev(X).requires_grad_(True)
    y = autograd.spmv(m, vals, x)
    (y * to_dev(G)).sum().backward()
    gx = x.grad.cpu().numpy()
    gv = vals.grad.cpu().numpy()
    h = 1e-6

    def loss(v, xx):
        return float((G * oracle.spmmv(A, xx, val=v)[0]).sum())

    rng = np.random.default_rng(0)
    for j, k in zip(rng.integers(0, A.nrows, 16), rng.integers(0, w, 16)):
        xp, xm = X.copy(), X.copy()
        xp[j, k] += h
        xm[j, k] -= h
        fd = (loss(A.val, xp) - loss(A.val, xm)) / (2 * h)
        assert abs(fd - gx[j, k]) <= 1e-6 * (1 + abs(fd))
    for p in rng.integers(0, A.nnz, 16):
        vp, vm = A.val.copy(), A.val.copy()
        vp[p] += h
        vm[p] -= h
        fd = (loss(vp, X) - loss(vm, X)) / (2 * h)
        assert abs(fd - gv[p]) <= 1e-6 * (1 + abs(fd))


@pytest.mark.slow
def test_powerlaw_full_size_fp32(cuda_ok):
    """N = 2^20, power-law row lengths in [1, 256] (exponent 2), float32 values
    and vectors, width 4: forward and backward against the oracle."""
    A, X, G = gen.workload_powerlaw()
    m = sellcs.SellMatrix(A, C=32, sigma=256, dtype="f32", with_transpose=True)
    vals = torch.tensor(A.val, dtype=torch.float32, device="cuda", requires_grad=True)
    x = to_dev(X, torch.float32).requires_grad_(True)
    y = autograd.spmv(m, vals, x)
    y.backward(to_dev(G, torch.float32))
    torch.cuda.synchronize()
    yr = oracle.spmmv(A, X)[0]
    maxlen = int(np.diff(A.rowptr).max())
    s = oracle.spmmv_scale(A, X) + np.abs(yr)
    assert_close(y.detach().double().cpu().numpy(), yr, s, 1.1 * (maxlen + 6) * U32, "forward")
    ref_dx = oracle.spmmv_transpose(A, G)
    collen = np.bincount(A.col, minlength=A.ncols)
    s_dx = oracle.spmmv_transpose(_abs(A), np.abs(G)) + np.abs(ref_dx)
    assert_close(x.grad.double().cpu().numpy(), ref_dx, s_dx, 1.1 * (collen.max() + 6) * U32, "dx")
    ref_dv = oracle.sampled_product(A, G, X)
    s_dv = oracle.sampled_product(A, np.abs(G), np.abs(X)) + np.abs(ref_dv)
    assert_close(vals.grad.double().cpu().numpy(), ref_dv, s_dv, 1.1 * 10 * U32, "dvals")


@pytest.mark.parametrize("C", [1, 4, 8])
def test_adjoint_threads_per_row(cuda_ok, C):
    A = gen.powerlaw(5000, seed=15)
    for w, xdt in ((1, "f64"), (4, "f32"), (2, "f64")):
        check_adjoint(A, w, C, 5000, xdt, seed=C)
