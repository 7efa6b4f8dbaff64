"""Pipelined products over host block vectors (sp_host_plan_*, sp_spmv_host):
several calls in flight on the plan's copy-in / product / copy-out streams
give, call by call, the same bits as sp_spmv on device copies of the same
inputs, and the oracle's product within the tolerance."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import sellcs
from tests.gpu_helpers import assert_close, to_dev, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def matrix():
    return gen.irregular_band(50_001, lmin=0, lmax=40, band=500, seed=41)


def _inputs(A, w, k, tdt):
    rng = np.random.default_rng(100 + k)
    X = rng.uniform(-1, 1, (A.ncols, w))
    Y0 = rng.uniform(-1, 1, (A.nrows, w))
    Z0 = rng.uniform(-1, 1, (A.nrows, w))
    if tdt == torch.float32:
        X, Y0, Z0 = (a.astype(np.float32).astype(np.float64) for a in (X, Y0, Z0))
    return X, Y0, Z0


@pytest.mark.parametrize("vdt,xdt", [("f64", "f64"), ("f32", "f32")])
@pytest.mark.parametrize("w", [1, 4, 33])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_plan_matches_device_product(cuda_ok, matrix, vdt, xdt, w, pinned):
    A = matrix
    tdt = torch.float64 if xdt == "f64" else torch.float32
    m = sellcs.SellMatrix(A, C=32, sigma=256, dtype=vdt)
    plan = sellcs.HostPlan(m, w, xdt)
    kw = dict(alpha=0.5, gamma=0.1, beta=1.0, dot_yy=True, dot_xy=True, delta=0.9, eta=0.1)
    calls = []
    for k in range(5):
        X, Y0, Z0 = _inputs(A, w, k, tdt)
        hx, hy, hz = (torch.from_numpy(a).to(tdt) for a in (X, Y0, Z0))
        oy, oz = torch.full_like(hy, float("nan")), torch.full_like(hz, float("nan"))
        od = torch.full((3 * w,), float("nan"), dtype=torch.float64)
        if pinned:
            hx, hy, hz, oy, oz, od = (t.pin_memory() for t in (hx, hy, hz, oy, oz, od))
        plan.spmv(hx, oy, y_in=hy, z_in=hz, z_out=oz, dot=od, **kw)
        calls.append((X, Y0, Z0, oy, oz, od))
    plan.sync()
    vals = oracle.round_values(A.val, vdt)
    for X, Y0, Z0, oy, oz, od in calls:
        x, y, z = to_dev(X, tdt), to_dev(Y0, tdt), to_dev(Z0, tdt)
        dot = torch.full((3 * w,), float("nan"), dtype=torch.float64, device="cuda")
        sellcs.spmv(m, x, y, alpha=0.5, gamma=0.1, beta=1.0, dot_yy=True, dot_xy=True, z=z, delta=0.9, eta=0.1,
                    dot=dot)
        torch.cuda.synchronize()
        assert torch.equal(oy, y.cpu()) and torch.equal(oz, z.cpu())
        d = od.numpy()
        assert np.array_equal(d[:2 * w], dot.cpu().numpy()[:2 * w]) and np.all(np.isnan(d[2 * w:]))
        yr, _, _ = oracle.spmmv(A, X, val=vals, alpha=0.5, gamma=0.1, beta=1.0, y0=Y0)
        s = oracle.spmmv_scale(A, X, val=vals, alpha=0.5, gamma=0.1, beta=1.0, y0=Y0)
        maxlen = int(np.diff(A.rowptr).max())
        tol = tol_for(vdt, xdt, maxlen)
        assert_close(oy.double().numpy(), yr, s + (np.abs(yr) if xdt == "f32" else 0), tol, "host plan y")
    plan.close()


def test_host_plan_rejects_bad_arguments(cuda_ok, matrix):
    m = sellcs.SellMatrix(matrix, C=32, sigma=1, dtype="f64")
    with pytest.raises(sellcs.SpError):
        sellcs.HostPlan(m, 2, "f32")  # float64 values need float64 vectors
    plan = sellcs.HostPlan(m, 1, "f64")
    x = np.zeros(matrix.ncols)
    y = np.zeros(matrix.nrows)
    with pytest.raises(sellcs.SpError):
        plan.spmv(x, y, beta=1.0)  # beta without y_in
    with pytest.raises(sellcs.SpError):
        plan.spmv(x, y, dot_yy=True)  # dots without a dot array
    plan.close()
