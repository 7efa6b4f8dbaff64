"""Scattered views of block vectors (Sec. "Dense matrices": a view selecting
columns with gaps between them), compact clones in either layout, copies
between views, and the product on scattered x, y, z: against the oracle on the
selected columns, with every column outside the views left untouched."""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import assert_close, dot_bound, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu
S = sellcs


def _view(t, layout):
    """View of an (n, W) CUDA tensor: row-major as is, column-major of t.t()
    storage (the tensor must then have unit row stride)."""
    return S.sp_dense_view(t, layout)


def _scattered(base, cols):
    c = np.ascontiguousarray(cols, np.int32)
    h = ct.c_void_p()
    S.check(S.lib().sp_dense_view_scattered(ct.byref(h), base, len(c), S._ptr(c)), "sp_dense_view_scattered")
    return h


def _block(n, W, layout, dtype, rng):
    a = rng.uniform(-1, 1, (n, W))
    t = torch.from_numpy(a).to("cuda", dtype)
    if layout == S.SP_COL_MAJOR:
        t = t.t().contiguous().t()
    return a, t


@pytest.mark.parametrize("layout", [S.SP_ROW_MAJOR, S.SP_COL_MAJOR])
@pytest.mark.parametrize("xdt", ["f64", "f32"])
def test_spmv_on_scattered_views(cuda_ok, layout, xdt):
    A = gen.irregular_band(3001, lmin=0, lmax=40, band=200, seed=17)
    rng = np.random.default_rng(4)
    tdt = torch.float64 if xdt == "f64" else torch.float32
    Wb = 7
    Xa, Xt = _block(A.nrows, Wb, layout, tdt, rng)
    Ya, Yt = _block(A.nrows, Wb, layout, tdt, rng)
    Za, Zt = _block(A.nrows, Wb, layout, tdt, rng)
    if xdt == "f32":
        Xa, Ya, Za = (a.astype(np.float32).astype(np.float64) for a in (Xa, Ya, Za))
    xc, yc, zc = [5, 0, 3], [6, 1, 2], [4, 2, 0]
    w = 3
    Y_before, Z_before = Yt.clone(), Zt.clone()
    m = S.SellMatrix(A, C=32, sigma=256, dtype=xdt)
    hX, hY, hZ = _view(Xt, layout), _view(Yt, layout), _view(Zt, layout)
    hx, hy, hz = _scattered(hX, xc), _scattered(hY, yc), _scattered(hZ, zc)
    dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device="cuda")
    gam = np.array([0.1, -0.2, 0.3])
    o, keep = S.make_opts(w, alpha=0.5, gamma=gam, beta=-1.5, dot_yy=True, dot_xy=True, dot_xx=True, z_handle=hz,
                          delta=0.9, eta=0.1, dot_ptr=S._ptr(dot))
    S.check(S.lib().sp_spmv(hy, m.handle, hx, ct.byref(o), S._stream(None)), "sp_spmv")
    torch.cuda.synchronize()
    X, Y0, Z0 = Xa[:, xc], Ya[:, yc], Za[:, zc]
    vals = oracle.round_values(A.val, xdt)
    yr, dr, zr = oracle.spmmv(A, X, val=vals, alpha=0.5, gamma=gam, beta=-1.5, y0=Y0, dot_yy=True, dot_xy=True,
                              dot_xx=True, delta=0.9, eta=0.1, z0=Z0)
    sc = oracle.spmmv_scale(A, X, val=vals, alpha=0.5, gamma=gam, beta=-1.5, y0=Y0)
    tol = tol_for(xdt, xdt, int(np.diff(A.rowptr).max()))
    if xdt == "f32":
        sc = sc + np.abs(yr)
    yg = Yt.double().cpu().numpy()
    zg = Zt.double().cpu().numpy()
    assert_close(yg[:, yc], yr, sc, tol, "scattered y")
    assert_close(zg[:, zc], zr, 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + sc), tol + (2 ** -24 if xdt == "f32" else 0),
                 "scattered z")
    d = dot.cpu().numpy()
    for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
        sl = slice(q * w, (q + 1) * w)
        assert_close(d[sl], dr[sl], dot_bound(name, yr, X, tol * sc, xdt, A.nrows), 1.0, f"scattered {name}")
    # columns outside the views are untouched, bit for bit
    other_y = [c for c in range(Wb) if c not in yc]
    other_z = [c for c in range(Wb) if c not in zc]
    assert torch.equal(Yt[:, other_y], Y_before[:, other_y])
    assert torch.equal(Zt[:, other_z], Z_before[:, other_z])
    for h in (hx, hy, hz, hX, hY, hZ):
        S.sp_dense_destroy(h)


def test_scattered_views_of_one_block_and_overlap(cuda_ok):
    """x and y as disjoint column sets of one block are accepted; sharing a
    column is aliasing (SP_ERR_ARG)."""
    A = gen.laplace3d(8)
    rng = np.random.default_rng(2)
    B = torch.from_numpy(rng.uniform(-1, 1, (A.nrows, 4))).cuda()
    B0 = B.clone()
    m = S.SellMatrix(A, C=32, sigma=1)
    hB = _view(B, S.SP_ROW_MAJOR)
    hx, hy = _scattered(hB, [0, 2]), _scattered(hB, [3, 1])
    o, _ = S.make_opts(2)
    S.check(S.lib().sp_spmv(hy, m.handle, hx, ct.byref(o), S._stream(None)), "sp_spmv")
    torch.cuda.synchronize()
    X = B0.cpu().numpy()[:, [0, 2]]
    yr, _, _ = oracle.spmmv(A, X)
    np.testing.assert_allclose(B.cpu().numpy()[:, [3, 1]], yr, rtol=1e-14, atol=1e-14)
    assert torch.equal(B[:, [0, 2]], B0[:, [0, 2]])
    hbad = _scattered(hB, [2, 1])  # shares column 2 with x
    assert S.lib().sp_spmv(hbad, m.handle, hx, ct.byref(o), S._stream(None)) == S.SP_ERR_ARG
    for h in (hx, hy, hbad, hB):
        S.sp_dense_destroy(h)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_clone_and_copy_between_layouts(cuda_ok, dtype):
    rng = np.random.default_rng(3)
    n, W = 1000, 70  # more columns than one copy launch takes (64)
    a = rng.uniform(-1, 1, (n, W))
    t = torch.from_numpy(a).to("cuda", dtype)
    hT = _view(t, S.SP_ROW_MAJOR)
    cols = list(rng.permutation(W)[:67])
    hs = _scattered(hT, cols)
    got = np.empty(67, np.int32)
    assert S.lib().sp_dense_columns(hs, S._ptr(got)) == 1
    np.testing.assert_array_equal(got, cols)
    L = S.lib()
    outs = []
    for lay in (S.SP_ROW_MAJOR, S.SP_COL_MAJOR):
        hc = ct.c_void_p()
        S.check(L.sp_dense_clone(ct.byref(hc), hs, lay, S._stream(None)), "sp_dense_clone")
        p, nr, nc, ld, dt, ly = ct.c_void_p(), ct.c_int64(), ct.c_int32(), ct.c_int64(), ct.c_int(), ct.c_int()
        S.check(L.sp_dense_data(hc, ct.byref(p), ct.byref(nr), ct.byref(nc), ct.byref(ld), ct.byref(dt),
                                ct.byref(ly)), "sp_dense_data")
        assert (nr.value, nc.value, ly.value) == (n, 67, lay)
        torch.cuda.synchronize()
        # read the clone back through a copy into a fresh row-major tensor
        back = torch.empty((n, 67), dtype=dtype, device="cuda")
        hb = _view(back, S.SP_ROW_MAJOR)
        S.check(L.sp_dense_copy(hb, hc, S._stream(None)), "sp_dense_copy")
        torch.cuda.synchronize()
        np.testing.assert_array_equal(back.cpu().numpy(), t.cpu().numpy()[:, cols])
        outs.append(hc)
        S.sp_dense_destroy(hb)
    # copy a scattered view onto another scattered view of a second block
    u = torch.zeros((n, W), dtype=dtype, device="cuda")
    hU = _view(u, S.SP_ROW_MAJOR)
    dcols = list(rng.permutation(W)[:67])
    hd = _scattered(hU, dcols)
    S.check(L.sp_dense_copy(hd, hs, S._stream(None)), "sp_dense_copy")
    torch.cuda.synchronize()
    un = u.cpu().numpy()
    np.testing.assert_array_equal(un[:, dcols], t.cpu().numpy()[:, cols])
    assert np.all(un[:, [c for c in range(W) if c not in dcols]] == 0)
    # a view and a differently scattered view of the same block overlap
    assert L.sp_dense_copy(_scattered(hT, cols[::-1]), hs, S._stream(None)) == S.SP_ERR_ARG
    for h in outs + [hs, hT, hd, hU]:
        S.sp_dense_destroy(h)


def test_scattered_views_refused_elsewhere(cuda_ok):
    L = S.lib()
    V = torch.zeros((100, 8), dtype=torch.float64, device="cuda")
    X = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    hV = _view(V, S.SP_ROW_MAJOR)
    hs = _scattered(hV, [0, 2, 4, 6])
    hX = _view(X, S.SP_ROW_MAJOR)
    assert L.sp_tsmttsm(hX, hs, hs, 1.0, 0.0, 0, S._stream(None)) == S.SP_ERR_ARG
    assert "scattered" in S.sp_last_error_detail()
    for h in (hs, hV, hX):
        S.sp_dense_destroy(h)
