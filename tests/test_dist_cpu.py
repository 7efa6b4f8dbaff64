"""Row-partitioned product, host side (no GPU): the partition, the per-process
plan (column split and halo compression), the send lists, the two-pass split
of the augmentation, and the whole distributed product on two gloo ranks.

The paper distributes the matrix row-wise (Sec. "Data parallelism"), with a
share per process (Sec. "Heterogeneous execution") and the remote column
indices compressed (the figure of the row-wise distribution, step 3).  The
checks here are brute force: sets and loops over small random matrices.  The
products in the last two tests are the oracle's, applied to the library's
split matrices with the library's split options; with integer data every sum
is exact, so the distributed result must equal the single product bit for
bit."""
import ctypes as ct
import json
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1507_08101_gb300 import dist, sellcs
from tests.test_oracle_format import random_csr
from workloads.generators import CSR

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _int_matrix(N, density, seed):
    rng = np.random.default_rng(seed)
    A = random_csr(N, N, density, rng)
    A.val = rng.integers(-3, 4, A.val.size).astype(np.float64)
    return A


def test_partition_nearest_boundaries():
    rng = np.random.default_rng(0)
    for trial in range(200):
        N = int(rng.integers(0, 60))
        lens = rng.integers(0, 9, N)
        rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
        P = int(rng.integers(1, 7))
        share = None if trial % 3 == 0 else rng.uniform(0, 3, P)
        if share is not None and share.sum() == 0:
            share[0] = 1.0
        by_nnz = bool(trial % 2)
        b = dist.partition(N, rowptr, P, share, by_nnz)
        assert b[0] == 0 and b[-1] == N and np.all(np.diff(b) >= 0)
        work = rowptr.astype(float) if by_nnz else np.arange(N + 1, dtype=float)
        sh = np.ones(P) if share is None else share
        cum = np.concatenate([[0], np.cumsum(sh)]) / sh.sum()
        for p in range(1, P):
            t = work[-1] * cum[p]
            # no admissible boundary (at or after the previous one) is nearer the target
            cand = np.arange(b[p - 1], N + 1)
            best = np.min(np.abs(work[cand] - t))
            assert abs(work[b[p]] - t) <= best + 1e-9, (trial, p, b, t)


def test_partition_by_rows_and_zero_share():
    b = dist.partition(100, None, 4, None, by_nnz=False)
    np.testing.assert_array_equal(b, [0, 25, 50, 75, 100])
    b = dist.partition(90, None, 3, [1.0, 0.0, 2.0], by_nnz=False)
    np.testing.assert_array_equal(b, [0, 30, 30, 90])  # the zero share gets no rows
    with pytest.raises(sellcs.SpError):
        dist.partition(10, None, 2, [0.0, 0.0], by_nnz=False)
    with pytest.raises(sellcs.SpError):
        dist.partition(3, np.array([0, 2, 1, 3]), 2, None, by_nnz=True)  # decreasing row pointers


def _plans(A, bounds):
    out = []
    for r in range(len(bounds) - 1):
        rp, gc, _ = dist.rows_of(A, bounds[r], bounds[r + 1])
        out.append(dist.DistPlan(A.nrows, bounds, r, rp, gc))
    return out


@pytest.mark.parametrize("P", [1, 2, 3, 5])
def test_plan_halo_and_split_brute_force(P):
    rng = np.random.default_rng(P)
    A = random_csr(97, 97, 0.08, rng)
    b = dist.partition(A.nrows, A.rowptr, P, rng.uniform(0.5, 2, P), True)
    for r, p in enumerate(_plans(A, b)):
        r0, r1 = b[r], b[r + 1]
        rp, gc, vv = dist.rows_of(A, r0, r1)
        remote = sorted({int(c) for c in gc if not (r0 <= c < r1)})
        halo, rc = p.halo()
        assert halo.tolist() == remote
        assert rc.tolist() == [sum(b[q] <= c < b[q + 1] for c in remote) for q in range(P)]
        assert rc[r] == 0
        info = p.info()
        assert info["nloc"] == r1 - r0 and info["nhalo"] == len(remote) and info["nsend"] == -1
        own = (gc >= r0) & (gc < r1)
        assert info["nnz_local"] == own.sum() and info["nnz_remote"] == (~own).sum()
        # compressed columns: own -> c - r0, remote -> nloc + position in the halo
        ce = p.columns()
        back = np.where(ce < r1 - r0, ce.astype(np.int64) + r0,
                        np.asarray(remote + [0], np.int64)[np.maximum(ce - (r1 - r0), 0)])
        np.testing.assert_array_equal(back, gc)
        # the split keeps every row's entries in order
        (rl, cl, vl), (rr, cr, vr) = p.split(vv)
        for i in range(r1 - r0):
            seg = slice(rp[i], rp[i + 1])
            m = ce[seg] < r1 - r0
            np.testing.assert_array_equal(cl[rl[i]:rl[i + 1]], ce[seg][m])
            np.testing.assert_array_equal(vl[rl[i]:rl[i + 1]], vv[seg][m])
            np.testing.assert_array_equal(cr[rr[i]:rr[i + 1]], ce[seg][~m])
            np.testing.assert_array_equal(vr[rr[i]:rr[i + 1]], vv[seg][~m])
        p.close()


def test_send_lists_and_errors():
    rng = np.random.default_rng(5)
    A = random_csr(40, 40, 0.15, rng)
    b = dist.partition(A.nrows, A.rowptr, 3, None, True)
    plans = _plans(A, b)
    halos = [p.halo()[0] for p in plans]
    for q, p in enumerate(plans):
        counts, lists = [], []
        for r in range(3):
            g = halos[r][(halos[r] >= b[q]) & (halos[r] < b[q + 1])] if r != q else np.zeros(0, np.int64)
            counts.append(g.size)
            lists.append(g)
        p.set_sends(counts, np.concatenate(lists))
        sc, sl = p.sends()
        assert sc.tolist() == counts
        np.testing.assert_array_equal(sl, np.concatenate(lists) - b[q])
        assert p.info()["nsend"] == sum(counts)
    p = plans[1]
    L = sellcs.lib()
    bad = [
        ([1, 0, 0], [b[0]]),              # a row of rank 0, not of rank 1
        ([0, 1, 0], [b[1]]),              # to itself
        ([2, 0, 0], [b[1] + 1, b[1]]),     # not ascending
    ]
    for counts, g in bad:
        if b[1] + 1 >= b[2]:
            continue
        with pytest.raises(sellcs.SpError) as e:
            p.set_sends(counts, g)
        assert e.value.code == sellcs.SP_ERR_ARG
    # plan inputs
    h = ct.c_void_p()
    rp = np.array([0, 1], np.int64)
    gc = np.array([7], np.int64)
    bnd = np.array([0, 1, 5], np.int64)
    assert L.sp_dist_plan_create(ct.byref(h), 6, 2, sellcs._ptr(bnd), 0, sellcs._ptr(rp),
                                 sellcs._ptr(gc)) == sellcs.SP_ERR_DIM  # bounds end at 5, not 6
    bnd = np.array([0, 1, 6], np.int64)
    assert L.sp_dist_plan_create(ct.byref(h), 6, 2, sellcs._ptr(bnd), 0, sellcs._ptr(rp),
                                 sellcs._ptr(gc)) == sellcs.SP_ERR_FORMAT  # column 7 outside [0, 6)
    assert L.sp_dist_plan_create(ct.byref(h), 6, 2, sellcs._ptr(bnd), 2, sellcs._ptr(rp),
                                 sellcs._ptr(gc)) == sellcs.SP_ERR_ARG  # no rank 2
    assert L.sp_dist_pack(None, None, None, None) == sellcs.SP_ERR_ARG
    assert L.sp_dist_spmv(None, None, None, None, None, None, None) == sellcs.SP_ERR_ARG


def _opts(w, *, alpha=None, gamma=None, beta=None, dots=(False, False, False), chain=None):
    zh = ct.c_void_p(0x10) if chain else None  # only copied by the split, never used here
    o, keep = sellcs.make_opts(w, alpha=alpha, gamma=gamma, beta=beta, dot_yy=dots[0], dot_xy=dots[1],
                               dot_xx=dots[2], z_handle=zh, delta=chain[0] if chain else None,
                               eta=chain[1] if chain else None, dot_ptr=ct.c_void_p(0x20) if any(dots) else None)
    return o, keep


def test_split_opts_flags():
    S = sellcs
    o, _keep = _opts(2, alpha=0.5, gamma=[0.1, 0.2], beta=-1.0, dots=(True, True, True), chain=(0.9, 0.1))
    o.flags |= S.SP_SPMV_DOT_HOST
    p1, p2 = dist.split_opts(o)
    late = S.SP_SPMV_DOT_ANY | S.SP_SPMV_DOT_HOST | S.SP_SPMV_CHAIN_AXPBY
    assert p1.flags == o.flags & ~late
    assert not p1.z and not p1.dot
    assert p2.flags == S.SP_SPMV_AXPBY | S.SP_SPMV_SCALE | late
    assert p2.alpha == 0.5 and p2.beta == 1.0 and p2.delta == 0.9 and p2.eta == 0.1
    assert p2.z == o.z and p2.dot == o.dot and not p2.gamma
    # plain y = A x: pass 2 adds the remote part to y (beta = 1, no scale)
    o, _ = _opts(1)
    p1, p2 = dist.split_opts(o)
    assert p1.flags == 0 and p2.flags == S.SP_SPMV_AXPBY and p2.beta == 1.0


def _oracle_kw(o, w):
    """The oracle's keywords for an sp_spmv_opts request."""
    S = sellcs
    f = o.flags
    kw = {}
    if f & S.SP_SPMV_SCALE:
        kw["alpha"] = o.alpha
    if f & S.SP_SPMV_SHIFT:
        kw["gamma"] = o.gamma[0]
    if f & S.SP_SPMV_VSHIFT:
        kw["gamma"] = [o.gamma[k] for k in range(w)]
    if f & S.SP_SPMV_AXPBY:
        kw["beta"] = o.beta
    kw.update(dot_yy=bool(f & S.SP_SPMV_DOT_YY), dot_xy=bool(f & S.SP_SPMV_DOT_XY),
              dot_xx=bool(f & S.SP_SPMV_DOT_XX))
    if f & S.SP_SPMV_CHAIN_AXPBY:
        kw.update(delta=o.delta, eta=o.eta)
    return kw


def _two_pass(plan, vals, x_ext, y0, z0, o, w):
    """One process's overlapped product with the oracle as the kernel:
    pass 1 over the local part, pass 2 over the remote part."""
    i = plan.info()
    n = i["nloc"]
    (rl, cl, vl), (rr, cr, vr) = plan.split(vals)
    Aloc = CSR(n, n, rl, cl, vl)
    Arem = CSR(n, n + i["nhalo"], rr, cr, vr)
    p1, p2 = dist.split_opts(o)
    k1 = _oracle_kw(p1, w)
    y1, _, _ = oracle.spmmv(Aloc, x_ext[:n], y0=y0 if "beta" in k1 else None, **k1)
    k2 = _oracle_kw(p2, w)
    y2, d2, z2 = oracle.spmmv(Arem, x_ext, y0=y1, z0=z0 if "delta" in k2 else None, **k2)
    return y2, d2, z2


REQS = [
    dict(alpha=2.0, gamma=1.0, beta=-1.0, dots=(True, True, True), chain=(1.0, 2.0)),
    dict(alpha=None, gamma=None, beta=None, dots=(True, False, False), chain=None),
    dict(alpha=-3.0, gamma=[1.0, -2.0, 0.0], beta=2.0, dots=(False, True, True), chain=(-1.0, 1.0)),
]


@pytest.mark.parametrize("P", [1, 2, 4])
@pytest.mark.parametrize("req", range(len(REQS)))
def test_two_pass_split_equals_single_product_exactly(P, req):
    """Integer data: every sum is exact, so the concatenated y, z and the
    summed dots of the parts equal the single product bit for bit."""
    A = _int_matrix(120, 0.06, 10 + P)
    w = 3
    rng = np.random.default_rng(P + 100 * req)
    X, Y0, Z0 = (rng.integers(-4, 5, (A.nrows, w)).astype(np.float64) for _ in range(3))
    kw = dict(REQS[req])
    o, _keep = _opts(w, **kw)
    b = dist.partition(A.nrows, A.rowptr, P, None, True)
    plans = _plans(A, b)
    ys, zs, ds = [], [], np.zeros(3 * w)
    for r, p in enumerate(plans):
        g, _ = p.halo()
        x_ext = np.concatenate([X[b[r]:b[r + 1]], X[g]])
        _, _, vv = dist.rows_of(A, b[r], b[r + 1])
        y, d, z = _two_pass(p, vv, x_ext, Y0[b[r]:b[r + 1]], Z0[b[r]:b[r + 1]], o, w)
        ys.append(y)
        zs.append(z)
        ds = ds + np.nan_to_num(d, nan=0.0)
    ok = _oracle_kw(o, w)
    yr, dr, zr = oracle.spmmv(A, X, y0=Y0 if "beta" in ok else None, z0=Z0 if "delta" in ok else None, **ok)
    np.testing.assert_array_equal(np.concatenate(ys), yr)
    if zr is not None:
        np.testing.assert_array_equal(np.concatenate(zs), zr)
    np.testing.assert_array_equal(ds[~np.isnan(dr)], dr[~np.isnan(dr)])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as tdist
    from paper_1507_08101_gb300 import dist as D
    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    comm = D.TorchComm()
    A = _int_matrix(150, 0.05, 77)  # every rank builds the same matrix and keeps its rows
    w = 2
    rng = np.random.default_rng(3)
    X, Y0, Z0 = (rng.integers(-4, 5, (A.nrows, w)).astype(np.float64) for _ in range(3))
    b = D.partition(A.nrows, A.rowptr, world, [1.0, 2.0][:world], True)
    r0, r1 = b[rank], b[rank + 1]
    rp, gc, vv = D.rows_of(A, r0, r1)
    plan = D.DistPlan(A.nrows, b, rank, rp, gc)
    plan.exchange_sends(comm)                       # all-to-all of the halo requests
    sc, sl = plan.sends()
    # the exchange of x itself: pack on the host (stand-in for sp_dist_pack, a
    # device gather), all-to-all through gloo into the halo rows
    g, rc = plan.halo()
    send = torch.from_numpy(np.ascontiguousarray(X[r0:r1][sl]))
    x_ext = torch.zeros((r1 - r0 + g.size, w), dtype=torch.float64)
    x_ext[:r1 - r0] = torch.from_numpy(X[r0:r1])
    comm.alltoallv(send, sc, x_ext[r1 - r0:], rc)
    o, _keep = _opts(w, alpha=2.0, gamma=1.0, beta=-1.0, dots=(True, True, False), chain=(1.0, 3.0))
    y, d, z = _two_pass(plan, vv, x_ext.numpy(), Y0[r0:r1], Z0[r0:r1], o, w)
    dt = torch.from_numpy(np.nan_to_num(d, nan=0.0))
    comm.allreduce_sum(dt)
    parts = [None] * world
    tdist.all_gather_object(parts, (y.tolist(), z.tolist()))
    tdist.destroy_process_group()
    if rank == 0:
        ok = _oracle_kw(o, w)
        yr, dr, zr = oracle.spmmv(A, X, y0=Y0, z0=Z0, **ok)
        res = {
            "halo_from_peer_exact": bool(np.array_equal(x_ext[r1 - r0:].numpy(), X[g])),
            "y_exact": bool(np.array_equal(np.concatenate([np.array(p[0]) for p in parts]), yr)),
            "z_exact": bool(np.array_equal(np.concatenate([np.array(p[1]) for p in parts]), zr)),
            "dots_exact": bool(np.array_equal(dt.numpy()[:2 * w], dr[:2 * w])),
            "sends": sc.tolist(),
        }
        with open(os.path.join(out_dir, "result.json"), "w") as f:
            json.dump(res, f)


def test_two_gloo_ranks_distributed_product(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_gloo_rank, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    res = json.load(open(tmp_path / "result.json"))
    assert res["halo_from_peer_exact"], res
    assert res["y_exact"] and res["z_exact"] and res["dots_exact"], res
    assert res["sends"][0] == 0 and res["sends"][1] > 0  # rank 0 sends to rank 1 only
