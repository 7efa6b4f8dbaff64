"""sp_spmv_noalloc, the entry point for callers that cannot allocate device
memory (their GPU memory is held by another allocator, or cudaMalloc is not
allowed where they run).

It is called through the C ABI, twice in a row per case (the shared static
scratch must be reset between calls), and its y, z and dots are compared

* with the float64 oracle, entry by entry, within the tolerances of the other
  parity tests (tests/gpu_helpers.py: tol_for for y and z, dot_bound for the
  dots), and
* with sp_spmv on the same matrix: y and z bit for bit (the same products are
  added in the same order in every row), the dots within the dot bound (the
  two assign rows to warps differently, so their dots add in another order).

Cases: every accepted precision pair, sorted and unsorted rows (sigma = 1
passes perm = NULL), chunk heights 32, 8 and 20, widths 1, 4 and 32 (the
widest, which sets the size of the static partial-sum array) with all dot
flags and the chain.

Collected last on purpose (file name), and self-contained, so it passes both
alone in a fresh process and after every other test."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs as F
from tests.gpu_helpers import assert_close, dot_bound, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu

ALL = (F.SP_SPMV_SCALE | F.SP_SPMV_VSHIFT | F.SP_SPMV_AXPBY | F.SP_SPMV_DOT_ANY | F.SP_SPMV_CHAIN_AXPBY)
PAIR = (F.SP_SPMV_SCALE | F.SP_SPMV_SHIFT | F.SP_SPMV_AXPBY | F.SP_SPMV_DOT_YY | F.SP_SPMV_DOT_XY
        | F.SP_SPMV_CHAIN_AXPBY)
# no fused reduction: wide row-major blocks then take the dynamic row order
# (its counters live beside the ticket in the static scratch)
NODOT = F.SP_SPMV_SCALE | F.SP_SPMV_VSHIFT | F.SP_SPMV_AXPBY | F.SP_SPMV_CHAIN_AXPBY
DT = {"f64": F.SP_F64, "f32": F.SP_F32, "bf16": F.SP_BF16}


@pytest.fixture(scope="module")
def matrix():
    return gen.irregular_band(20011, lmin=0, lmax=48, band=700, seed=31)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def _noalloc(m, A, e, x, y, z, w, flags, vdt, xdt, gam, alpha, beta, delta, eta, dot, use_perm):
    val, col = _dev(e["val_stored"]), _dev(e["col"])
    chunkptr, slotlen = _dev(e["chunkptr"]), _dev(e["slotlen"])
    perm = _dev(e["perm"]) if use_perm else None
    g = np.ascontiguousarray(gam, np.float64)
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = F.lib().sp_spmv_noalloc(ct.c_void_p(val.data_ptr()), DT[vdt], ct.c_void_p(col.data_ptr()),
                                 ct.c_void_p(chunkptr.data_ptr()), ct.c_void_p(slotlen.data_ptr()),
                                 ct.c_void_p(perm.data_ptr()) if perm is not None else None,
                                 A.nrows, A.ncols, m.info()["C"],
                                 ct.c_void_p(x.data_ptr()), w, ct.c_void_p(y.data_ptr()), w,
                                 ct.c_void_p(z.data_ptr()), w, w, DT[xdt], flags, alpha, beta,
                                 g.ctypes.data_as(ct.POINTER(ct.c_double)), delta, eta,
                                 ct.c_void_p(dot.data_ptr()), stream)
    assert rc == 0, F.sp_last_error_detail()
    # keep the device copies alive until the call has run
    torch.cuda.synchronize()


def _stored_values(m, vdt):
    """SELL arrays of the matrix with the values in the stored precision."""
    e = m.export_sell()
    v = e["val"]
    if vdt == "f64":
        e["val_stored"] = v
    elif vdt == "f32":
        e["val_stored"] = v.astype(np.float32)
    else:  # bf16: the exported values are exact bf16 numbers widened to f64
        e["val_stored"] = torch.from_numpy(v).to(torch.bfloat16).view(torch.int16).numpy()
    return e


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f64"), ("bf16", "f64"), ("f32", "f32"),
                                     ("bf16", "f32")])
@pytest.mark.parametrize("C,sigma", [(32, 256), (32, 1), (8, 64), (20, 1)])
def test_noalloc_matches_oracle_and_sp_spmv_twice(cuda_ok, matrix, vdt, xdt, C, sigma):
    A = matrix
    m = F.SellMatrix(A, C=C, sigma=sigma, dtype=vdt)
    e = _stored_values(m, vdt)
    vals = oracle.round_values(A.val, vdt)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    tol = tol_for(vdt, xdt, int(np.diff(A.rowptr).max()))
    rng = np.random.default_rng(7 + C + sigma)
    cases = [(32, ALL), (16, NODOT), (4, ALL), (1, PAIR), (16, NODOT)]
    for call, (w, flags) in enumerate(cases + cases[:1]):  # the widest case again as the last call
        X, Y0, Z0 = (rng.uniform(-1, 1, (A.nrows, w)) for _ in range(3))
        if xdt == "f32":
            X, Y0, Z0 = (v.astype(np.float32).astype(np.float64) for v in (X, Y0, Z0))
        gam = rng.uniform(-1, 1, w) if flags & F.SP_SPMV_VSHIFT else np.array([0.3])
        gam_o = gam if flags & F.SP_SPMV_VSHIFT else float(gam[0])
        alpha, beta, delta, eta = 0.5, -1.5, 0.9, 0.1
        dflags = dict(dot_yy=bool(flags & F.SP_SPMV_DOT_YY), dot_xy=bool(flags & F.SP_SPMV_DOT_XY),
                      dot_xx=bool(flags & F.SP_SPMV_DOT_XX))
        # the no-allocation entry point
        x, y, z = _dev(X, tdt), _dev(Y0, tdt), _dev(Z0, tdt)
        dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device="cuda")
        _noalloc(m, A, e, x, y, z, w, flags, vdt, xdt, gam, alpha, beta, delta, eta, dot, use_perm=sigma > 1)
        yn, zn, dn = (t.double().cpu().numpy() for t in (y, z, dot))
        # the oracle
        yr, dr, zr = oracle.spmmv(A, X, val=vals, alpha=alpha, gamma=gam_o, beta=beta, y0=Y0, delta=delta, eta=eta,
                                  z0=Z0, **dflags)
        sc = oracle.spmmv_scale(A, X, val=vals, alpha=alpha, gamma=gam_o, beta=beta, y0=Y0)
        if xdt == "f32":
            sc = sc + np.abs(yr)
        what = f"call {call} w={w} {vdt}/{xdt} C={C} sigma={sigma}"
        assert_close(yn, yr, sc, tol, f"{what}: y vs oracle")
        zsc = 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + sc)
        assert_close(zn, zr, zsc, tol + (2 ** -24 if xdt == "f32" else 0), f"{what}: z vs oracle")
        for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
            sl = slice(q * w, (q + 1) * w)
            if flags & (F.SP_SPMV_DOT_YY << q):
                assert_close(dn[sl], dr[sl], dot_bound(name, yr, X, tol * sc, xdt, A.nrows), 1.0,
                             f"{what}: {name} vs oracle")
            else:
                assert np.all(np.isnan(dn[sl])), f"{what}: unrequested {name} written"
        # the existing entry point on the same inputs
        x2, y2, z2 = _dev(X, tdt), _dev(Y0, tdt), _dev(Z0, tdt)
        d2 = F.spmv(m, x2, y2, alpha=alpha, gamma=gam_o, beta=beta, z=z2, delta=delta, eta=eta, **dflags)
        torch.cuda.synchronize()
        assert torch.equal(y2, y), f"{what}: y differs from sp_spmv"
        assert torch.equal(z2, z), f"{what}: z differs from sp_spmv"
        d2 = d2.cpu().numpy() if d2 is not None else None  # None: no dot requested
        for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
            sl = slice(q * w, (q + 1) * w)
            if flags & (F.SP_SPMV_DOT_YY << q):
                bound = 2 * dot_bound(name, yr, X, tol * sc, xdt, A.nrows)
                assert_close(dn[sl], d2[sl], bound, 1.0, f"{what}: {name} vs sp_spmv")


def test_noalloc_rejects_too_wide_block(cuda_ok):
    L = F.lib()
    rc = L.sp_spmv_noalloc(None, F.SP_F64, None, None, None, None, 10, 10, 32, None, 64, None, 64, None, 64,
                           F.SP_NOALLOC_MAX_W + 1,
                           F.SP_F64, 0, 1.0, 0.0, None, 0.0, 1.0, None, None)
    assert rc == F.SP_ERR_UNSUPPORTED
    assert "SP_NOALLOC_MAX_W" in F.sp_last_error_detail()
