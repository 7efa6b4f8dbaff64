"""Autotuner: host-side candidate logic (CPU) and a tuned batch on the GPU that
multiplies exactly like the untuned one and feeds the CG solver."""
import numpy as np
import pytest

from paper_1507_08101_gb300 import autotune
from workloads import generators as gen


def test_lane_candidates():
    assert autotune.lane_candidates(1, 4) == [1]
    assert autotune.lane_candidates(8, 4) == [1, 2, 4]
    assert autotune.lane_candidates(8, 8) == [1, 2]
    assert autotune.lane_candidates(6, 4) == [1, 2]
    assert autotune.lane_candidates(3, 8) == [1]
    assert autotune.lane_candidates(4, 8) == [1, 2]
    for w in range(1, 9):
        for xs in (4, 8):
            for c in autotune.lane_candidates(w, xs):
                assert w % c == 0 and (w * xs) % min(16, c * xs) == 0 and c <= (2 if xs == 8 else 4)


def test_signature_is_structural():
    a = gen.laplace2d(20)
    b = gen.laplace2d(20, shift=5.0)  # same pattern, other values
    c = gen.laplace2d(21)
    assert autotune.signature(a, 2, "f32") == autotune.signature(b, 2, "f32")
    assert autotune.signature(a, 2, "f32") != autotune.signature(a, 3, "f32")
    assert autotune.signature(a, 2, "f32") != autotune.signature(c, 2, "f32")


@pytest.mark.gpu
def test_tuned_batch_runs_and_caches(cuda_ok, tmp_path):
    import torch
    from paper_1507_08101_gb300 import sellcs
    mats = [gen.laplace2d(s, 0.01) for s in (40, 64, 40)]
    widths = [2, 5, 2]
    cache = str(tmp_path / "tune.json")
    cfg = autotune.tune_batch(mats, widths, cache_path=cache, reps=5, sigmas=(1, 32))
    assert cfg[0] == cfg[2]  # same structure and width: tuned once
    for c, w in zip(cfg, widths):
        assert c["C"] in autotune.C_CANDIDATES and c["sigma"] in (1, 32) and w % c["cpl"] == 0
    again = autotune.tune_batch(mats, widths, cache_path=cache, reps=5, sigmas=(1, 32))
    assert again == cfg
    S = [sellcs.SellMatrix(A, C=c["C"], sigma=c["sigma"], dtype="f32") for A, c in zip(mats, cfg)]
    xs = [torch.rand(A.nrows, w, dtype=torch.float32, device="cuda") for A, w in zip(mats, widths)]
    y1 = [torch.empty_like(x) for x in xs]
    y2 = [torch.empty_like(x) for x in xs]
    b1 = sellcs.Batch(S, widths, cols_per_lane=[c["cpl"] for c in cfg], vec_dtype="f32")
    b1.bind(xs, y1)
    b1.spmv()
    b2 = sellcs.Batch(S, widths, vec_dtype="f32")
    b2.bind(xs, y2)
    b2.spmv()
    torch.cuda.synchronize()
    import oracle
    for a, b, A, c, x in zip(y1, y2, mats, cfg, xs):
        if c["C"] == 32:
            # one lane per row in every layout: the same sums, bit for bit
            assert torch.equal(a, b)
        else:
            # rows split over several lanes add their products in an order that
            # depends on the lane layout: equal within the float32 bound
            X = x.double().cpu().numpy()
            sc = oracle.spmmv_scale(A, X, val=oracle.round_values(A.val, "f32"))
            tol = 2 * 1.1 * (int(np.diff(A.rowptr).max()) + 6) * 2.0 ** -24
            d = np.abs(a.double().cpu().numpy() - b.double().cpu().numpy())
            assert np.all(d <= tol * sc + 1e-30)


@pytest.mark.gpu
def test_joint_tuning(cuda_ok, tmp_path):
    mats = [gen.laplace2d(s, 0.01) for s in (30, 50, 70)]
    widths = [1, 4, 8]
    cfg = autotune.tune_batch_joint(mats, widths, cache_path=str(tmp_path / "j.json"), reps=5,
                                    Cs=(16, 32), sigmas=(1, 32))
    assert len({(c["C"], c["sigma"]) for c in cfg}) == 1
    for c, w in zip(cfg, widths):
        assert w % c["cpl"] == 0 and c["cpl"] <= 4
    assert autotune.tune_batch_joint(mats, widths, cache_path=str(tmp_path / "j.json"), reps=5,
                                     Cs=(16, 32), sigmas=(1, 32)) == cfg


@pytest.mark.gpu
def test_tune_spmv_forward_and_adjoint(cuda_ok, tmp_path):
    """The single-matrix tuner returns a candidate configuration, caches it, and
    the matrix built with it gives the oracle's product and adjoint."""
    import torch
    import oracle
    from paper_1507_08101_gb300 import sellcs
    from tests.gpu_helpers import to_dev
    A = gen.powerlaw(20000, seed=17)
    cache = str(tmp_path / "tune.json")
    cfg = autotune.tune_spmv(A, 4, "f32", "f32", with_transpose=True, cache_path=cache, reps=3, Cs=(8, 32))
    assert cfg["C"] in (8, 32) and cfg["sigma"] in (1, 256, A.nrows) and cfg["order"] in autotune.SPMV_ORDERS
    assert autotune.tune_spmv(A, 4, "f32", "f32", with_transpose=True, cache_path=cache, reps=3,
                              Cs=(8, 32)) == cfg
    m = sellcs.SellMatrix(A, C=cfg["C"], sigma=cfg["sigma"], dtype="f32", with_transpose=True, order=cfg["order"])
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (A.ncols, 4)).astype(np.float32).astype(np.float64)
    G = rng.uniform(-1, 1, (A.nrows, 4)).astype(np.float32).astype(np.float64)
    x, g = to_dev(X, torch.float32), to_dev(G, torch.float32)
    y = torch.empty_like(x)
    sellcs.spmv(m, x, y)
    dx, dv = torch.empty_like(x), torch.empty(A.nnz, dtype=torch.float32, device="cuda")
    sellcs.spmv_adjoint(m, g, x=x, dx=dx, dvals=dv)
    torch.cuda.synchronize()
    vals = oracle.round_values(A.val, "f32")
    yr, _, _ = oracle.spmmv(A, X, val=vals)
    dxr = oracle.spmmv_transpose(A, G, val=vals)
    dvr = oracle.sampled_product(A, G, X)
    maxlen = int(np.diff(A.rowptr).max())
    tol = 1.1 * (maxlen + 6) * 2.0 ** -24
    s = oracle.spmmv_scale(A, X, val=vals)
    assert np.all(np.abs(y.double().cpu().numpy() - yr) <= tol * (s + np.abs(yr)) + 1e-30)
    sT = np.abs(oracle.spmmv_transpose(A, np.abs(G), val=np.abs(vals)))
    assert np.all(np.abs(dx.double().cpu().numpy() - dxr) <= 2 * tol * (sT + np.abs(dxr)) + 1e-30)
    np.testing.assert_allclose(dv.double().cpu().numpy(), dvr, rtol=tol * 8, atol=tol * 8)
