"""sp_spmv_noalloc, the entry point for callers that cannot allocate device
memory (their GPU memory is held by another allocator, or cudaMalloc is not
allowed where they run): called through the C ABI twice in a row, its output
must match sp_spmv's on the same inputs within the tolerance of the other
parity tests (1e-12 relative to the magnitude scale for float64).

Collected last on purpose (file name), and self-contained, so it passes both
alone in a fresh process and after every other test."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from workloads import generators as gen

pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def test_noalloc_matches_sp_spmv_twice(cuda_ok):
    A = gen.irregular_band(20011, lmin=0, lmax=48, band=700, seed=31)
    m = sellcs.SellMatrix(A, C=32, sigma=256)
    e = m.export_sell()
    val, col = _dev(e["val"]), _dev(e["col"])
    chunkptr, slotlen, perm = _dev(e["chunkptr"]), _dev(e["slotlen"]), _dev(e["perm"])
    L = sellcs.lib()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    F = sellcs
    cases = [
        (4, F.SP_SPMV_SCALE | F.SP_SPMV_VSHIFT | F.SP_SPMV_AXPBY | F.SP_SPMV_DOT_ANY | F.SP_SPMV_CHAIN_AXPBY),
        (1, F.SP_SPMV_SCALE | F.SP_SPMV_SHIFT | F.SP_SPMV_AXPBY | F.SP_SPMV_DOT_YY | F.SP_SPMV_DOT_XY
         | F.SP_SPMV_CHAIN_AXPBY),
    ]
    rng = np.random.default_rng(7)
    for call, (w, flags) in enumerate(cases):
        X = rng.uniform(-1, 1, (A.nrows, w))
        Y0 = rng.uniform(-1, 1, (A.nrows, w))
        Z0 = rng.uniform(-1, 1, (A.nrows, w))
        gam = rng.uniform(-1, 1, w) if flags & F.SP_SPMV_VSHIFT else np.array([0.3])
        alpha, beta, delta, eta = 0.5, -1.5, 0.9, 0.1
        # existing entry point
        x = _dev(X)
        y_ref, z_ref = _dev(Y0), _dev(Z0)
        d_ref = sellcs.spmv(m, x, y_ref, alpha=alpha, gamma=gam if w > 1 else float(gam[0]), beta=beta,
                            dot_yy=bool(flags & F.SP_SPMV_DOT_YY), dot_xy=bool(flags & F.SP_SPMV_DOT_XY),
                            dot_xx=bool(flags & F.SP_SPMV_DOT_XX), z=z_ref, delta=delta, eta=eta)
        # the no-allocation entry point
        y, z = _dev(Y0), _dev(Z0)
        dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device="cuda")
        g = np.ascontiguousarray(gam, np.float64)
        rc = L.sp_spmv_noalloc(ct.c_void_p(val.data_ptr()), F.SP_F64, ct.c_void_p(col.data_ptr()),
                               ct.c_void_p(chunkptr.data_ptr()), ct.c_void_p(slotlen.data_ptr()),
                               ct.c_void_p(perm.data_ptr()), A.nrows, A.ncols, 32,
                               ct.c_void_p(x.data_ptr()), w, ct.c_void_p(y.data_ptr()), w,
                               ct.c_void_p(z.data_ptr()), w, w, F.SP_F64, flags, alpha, beta,
                               g.ctypes.data_as(ct.POINTER(ct.c_double)), delta, eta,
                               ct.c_void_p(dot.data_ptr()), stream)
        assert rc == 0, sellcs.sp_last_error_detail()
        torch.cuda.synchronize()
        s = oracle.spmmv_scale(A, X, alpha=alpha, gamma=gam if w > 1 else float(gam[0]), beta=beta, y0=Y0)
        yn, yr = y.cpu().numpy(), y_ref.cpu().numpy()
        assert np.all(np.abs(yn - yr) <= 1e-12 * s + 1e-300), f"call {call}: y differs"
        zs = 0.9 * np.abs(Z0) + 0.1 * s
        assert np.all(np.abs(z.cpu().numpy() - z_ref.cpu().numpy()) <= 1e-12 * zs + 1e-300), f"call {call}: z"
        dn, dr = dot.cpu().numpy(), d_ref.cpu().numpy()
        for q in range(3):
            sl = slice(q * w, (q + 1) * w)
            if flags & (F.SP_SPMV_DOT_YY << q):
                np.testing.assert_allclose(dn[sl], dr[sl], rtol=1e-12, atol=1e-12, err_msg=f"call {call} dot {q}")
            else:
                assert np.all(np.isnan(dn[sl]))


def test_noalloc_rejects_too_wide_block(cuda_ok):
    L = sellcs.lib()
    rc = L.sp_spmv_noalloc(None, sellcs.SP_F64, None, None, None, None, 10, 10, 32, None, 64, None, 64, None, 64,
                           sellcs.SP_NOALLOC_MAX_W + 1,
                           sellcs.SP_F64, 0, 1.0, 0.0, None, 0.0, 1.0, None, None)
    assert rc == sellcs.SP_ERR_UNSUPPORTED
    assert "SP_NOALLOC_MAX_W" in sellcs.sp_last_error_detail()
