"""Row-partitioned product on one GPU: every part of the partition runs in
this process (dist.LocalWorld), with the library's halo pack, the
device-to-device halo copies and the library's product (the two-pass
overlapped form or the one-pass form over the extended columns).  The
concatenated y, z and the summed dots are compared with the oracle's single
product entry by entry; with integer data they must equal the single-GPU
product bit for bit.  The parts run one after another: no kernel waits for
another part's kernel."""
import numpy as np
import pytest
import torch

import oracle
from paper_1507_08101_gb300 import dist, sellcs
from tests.gpu_helpers import assert_close, dot_bound, tol_for
from workloads import generators as gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def band():
    return gen.irregular_band(12007, lmin=0, lmax=40, band=600, seed=41)


def _run(world, X, Y0, Z0, kw, w, tdt):
    xs = world.scatter(torch.from_numpy(X).to(tdt))
    ys, zs = [], []
    for r, m in enumerate(world.mats):
        r0, r1 = world.bounds[r], world.bounds[r + 1]
        ys.append(torch.from_numpy(Y0[r0:r1]).to("cuda", tdt).contiguous())
        zs.append(torch.from_numpy(Z0[r0:r1]).to("cuda", tdt).contiguous())
    d = world.spmv(xs, ys, zs if "delta" in kw else None, **kw)
    torch.cuda.synchronize()
    y = torch.cat(ys).double().cpu().numpy()
    z = torch.cat(zs).double().cpu().numpy()
    return y, z, (d.cpu().numpy() if d is not None else None), xs


@pytest.mark.parametrize("mode", ["overlap", "no_overlap"])
@pytest.mark.parametrize("P", [1, 2, 3, 5])
@pytest.mark.parametrize("w", [1, 4])
def test_partitioned_matches_oracle(cuda_ok, band, mode, P, w):
    A = band
    rng = np.random.default_rng(P * 10 + w)
    X, Y0, Z0 = (rng.uniform(-1, 1, (A.nrows, w)) for _ in range(3))
    gam = rng.uniform(-1, 1, w) if w > 1 else 0.3
    share = rng.uniform(0.5, 2.0, P)
    world = dist.LocalWorld(A, P, C=32, sigma=256, mode=mode, share=share)
    kw = dict(alpha=0.5, gamma=gam, beta=-1.5, dot_yy=True, dot_xy=True, dot_xx=True, delta=0.9, eta=0.1)
    y, z, d, xs = _run(world, X, Y0, Z0, kw, w, torch.float64)
    # the halo rows hold exactly the x rows of the compressed remote columns
    for r, p in enumerate(world.plans):
        g, _ = p.halo()
        np.testing.assert_array_equal(xs[r][world.mats[r].nloc:].cpu().numpy(), X[g])
    ok = dict(alpha=0.5, gamma=gam, beta=-1.5, y0=Y0, dot_yy=True, dot_xy=True, dot_xx=True, delta=0.9, eta=0.1,
              z0=Z0)
    yr, dr, zr = oracle.spmmv(A, X, **ok)
    sc = oracle.spmmv_scale(A, X, alpha=0.5, gamma=gam, beta=-1.5, y0=Y0)
    # two passes: the local pass's rounded y is added to the remote part, one
    # more rounding of a term bounded by the same scale
    tol = 2 * tol_for("f64", "f64", 0)
    assert_close(y, yr, sc, tol, f"P={P} {mode} y")
    assert_close(z, zr, 0.9 * np.abs(Z0) + 0.1 * (np.abs(yr) + sc), tol, f"P={P} {mode} z")
    for q, name in enumerate(["dot_yy", "dot_xy", "dot_xx"]):
        sl = slice(q * w, (q + 1) * w)
        # P parts summed on the host in part order: P more float64 additions
        b = dot_bound(name, yr, X, tol * sc, "f64", A.nrows + P)
        assert_close(d[sl], dr[sl], b, 1.0, f"P={P} {mode} {name}")
    for m in world.mats:
        m.close()


@pytest.mark.parametrize("mode", ["overlap", "no_overlap"])
def test_partitioned_integer_data_bit_exact(cuda_ok, mode):
    """Integer matrix and vectors: every partial sum is exact, so the parts'
    y, z and summed dots equal the single-GPU product's bits."""
    rng = np.random.default_rng(9)
    A = gen.irregular_band(5003, lmin=0, lmax=30, band=300, seed=43)
    A.val = rng.integers(-3, 4, A.val.size).astype(np.float64)
    w = 2
    X, Y0, Z0 = (rng.integers(-4, 5, (A.nrows, w)).astype(np.float64) for _ in range(3))
    kw = dict(alpha=2.0, gamma=[1.0, -1.0], beta=-1.0, dot_yy=True, dot_xy=True, dot_xx=True, delta=1.0, eta=2.0)
    world = dist.LocalWorld(A, 4, C=32, sigma=32, mode=mode)
    y, z, d, _ = _run(world, X, Y0, Z0, kw, w, torch.float64)
    m = sellcs.SellMatrix(A, C=32, sigma=32)
    xg, yg, zg = (torch.from_numpy(a).cuda() for a in (X, Y0.copy(), Z0.copy()))
    dg = sellcs.spmv(m, xg, yg, z=zg, **kw)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(y, yg.cpu().numpy())
    np.testing.assert_array_equal(z, zg.cpu().numpy())
    np.testing.assert_array_equal(d, dg.cpu().numpy())


def test_partitioned_float32(cuda_ok, band):
    A = band
    rng = np.random.default_rng(5)
    w = 4
    X, Y0, Z0 = (rng.uniform(-1, 1, (A.nrows, w)).astype(np.float32).astype(np.float64) for _ in range(3))
    world = dist.LocalWorld(A, 3, C=32, sigma=1, dtype="f32", mode="overlap")
    kw = dict(alpha=0.5, beta=1.0, dot_yy=True, dot_xy=True)
    y, _, d, _ = _run(world, X, Y0, Z0, kw, w, torch.float32)
    vals = oracle.round_values(A.val, "f32")
    yr, dr, _ = oracle.spmmv(A, X, val=vals, alpha=0.5, beta=1.0, y0=Y0, dot_yy=True, dot_xy=True)
    sc = oracle.spmmv_scale(A, X, val=vals, alpha=0.5, beta=1.0, y0=Y0) + np.abs(yr)
    tol = 2 * tol_for("f32", "f32", int(np.diff(A.rowptr).max()))
    assert_close(y, yr, sc, tol, "f32 y")
    for q, name in enumerate(["dot_yy", "dot_xy"]):
        sl = slice(q * w, (q + 1) * w)
        assert_close(d[sl], dr[sl], dot_bound(name, yr, X, tol * sc, "f32", A.nrows + 3), 1.0, f"f32 {name}")


def test_empty_part_and_no_halo(cuda_ok):
    """A zero share gives a part with no rows; a block-diagonal matrix gives
    parts without a halo (the remote pass still applies the dots and chain)."""
    n = 64
    rp = np.arange(n + 1, dtype=np.int64)
    A = gen.CSR(n, n, rp, np.arange(n, dtype=np.int32), np.full(n, 2.0))
    rng = np.random.default_rng(1)
    X, Y0, Z0 = (rng.uniform(-1, 1, (n, 1)) for _ in range(3))
    world = dist.LocalWorld(A, 3, share=[1.0, 0.0, 1.0])
    assert world.bounds[1] == world.bounds[2]
    assert all(p.info()["nhalo"] == 0 for p in world.plans)
    kw = dict(alpha=0.5, beta=1.0, dot_yy=True, delta=0.5, eta=1.0)
    y, z, d, _ = _run(world, X, Y0, Z0, kw, 1, torch.float64)
    yr, dr, zr = oracle.spmmv(A, X, alpha=0.5, beta=1.0, y0=Y0, dot_yy=True, delta=0.5, eta=1.0, z0=Z0)
    np.testing.assert_array_equal(y, yr)  # y = x + y0 exactly: 0.5 * 2 x + y0
    assert_close(z, zr, np.abs(zr) + 1, 1e-15, "z")
    assert_close(d[:1], dr[:1], dot_bound("dot_yy", yr, X, 1e-12 * np.abs(yr), "f64", n + 3), 1.0, "dot_yy")
