"""Autotuner of the SpMMV launch configuration.

For the batched kernel it picks the SELL chunk height C, the sort window sigma
and the lane layout (columns per lane CPL, hence G = WP / CPL lanes per column
group and, through C, the threads per row T) by timing candidates on the GPU
with CUDA events: either jointly for a whole batch (:func:`tune_batch_joint`:
every candidate batch is built with sp_mat_create_csr and multiplied by one
sp_batch launch, the kernel the solver runs) or per matrix (:func:`tune_batch`:
each matrix through a one-matrix sp_batch).  For a single matrix multiplied by
sp_spmv (and differentiated by sp_spmv_adjoint) :func:`tune_spmv` picks C,
sigma and the work order (moving front or contiguous ranges).  Results are
cached in a JSON file under a structural signature of the matrix (size,
nonzeros, row-length histogram) and the block width, so equal structures are
tuned once.

This module only orchestrates calls into the CUDA library; the timed work is
the library's kernels.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

from . import sellcs

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sellcs_autotune.json")
C_CANDIDATES = (8, 16, 32)
SIGMA_CANDIDATES = (1, 32, 256, 1024)


def signature(A, w: int, dtype: str) -> str:
    lens = np.diff(np.asarray(A.rowptr))
    h = hashlib.sha1()
    h.update(np.bincount(lens).astype(np.int64).tobytes())
    h.update(np.asarray(lens[: min(4096, lens.size)], np.int64).tobytes())
    return f"{A.nrows}x{A.ncols}:{A.nnz}:w{w}:{dtype}:{h.hexdigest()[:16]}"


def lane_candidates(w: int, xsize: int):
    """Columns per lane that divide w, keep every row 8/16-byte aligned and do
    not exceed the batched kernel's widest lane (2 doubles or 4 floats)."""
    wp = 1
    while wp < w:
        wp <<= 1
    out = []
    c = 1
    while c <= min(wp, 2 if xsize == 8 else 4):
        if w % c == 0 and (w * xsize) % min(16, c * xsize) == 0:
            out.append(c)
        c <<= 1
    return out


def _time_batch(batch, reps: int) -> float:
    import torch
    for _ in range(3):
        batch.spmv()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.spmv()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) * 1e3 / reps  # microseconds


def tune_matrix(A, w: int, dtype: str = "f32", vec_dtype: str = "f32", reps: int = 20,
                Cs=C_CANDIDATES, sigmas=SIGMA_CANDIDATES) -> dict:
    import torch
    tdt = torch.float32 if vec_dtype == "f32" else torch.float64
    xs = 4 if vec_dtype == "f32" else 8
    x = torch.rand(A.ncols, w, dtype=tdt, device="cuda")
    y = torch.empty(A.nrows, w, dtype=tdt, device="cuda")
    best = None
    for C in Cs:
        for sigma in sigmas:
            if sigma > 1 and sigma < C:
                continue
            m = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=dtype)
            for cpl in lane_candidates(w, xs):
                b = sellcs.Batch([m], [w], cols_per_lane=[cpl], vec_dtype=vec_dtype)
                b.bind([x], [y])
                us = _time_batch(b, reps)
                b.close()
                if best is None or us < best["us"]:
                    best = {"C": C, "sigma": sigma, "cpl": cpl, "us": round(us, 3)}
            m.close()
    return best


LANE_POLICIES = ("widest", "narrowest", "middle")


def _policy_cpl(w: int, xsize: int, policy: str) -> int:
    c = lane_candidates(w, xsize)
    return c[-1] if policy == "widest" else (c[0] if policy == "narrowest" else c[len(c) // 2])


def tune_batch_joint(mats, widths, dtype: str = "f32", vec_dtype: str = "f32",
                     cache_path: str | None = DEFAULT_CACHE, reps: int = 20, Cs=C_CANDIDATES,
                     sigmas=SIGMA_CANDIDATES):
    """One (C, sigma, lane policy) for the whole batch, chosen by timing the
    batched launch itself (what the solver runs), so small matrices whose solo
    launches are latency-bound do not decide by noise.  Returns the per-matrix
    list of {C, sigma, cpl, us} (us: the batch time)."""
    import torch
    key = "batch:" + hashlib.sha1("|".join(signature(A, w, dtype) for A, w in zip(mats, widths)).encode()
                                  ).hexdigest()[:20]
    cache = _load_cache(cache_path)
    if key not in cache:
        tdt = torch.float32 if vec_dtype == "f32" else torch.float64
        xs = 4 if vec_dtype == "f32" else 8
        xv = [torch.rand(A.ncols, w, dtype=tdt, device="cuda") for A, w in zip(mats, widths)]
        yv = [torch.empty(A.nrows, w, dtype=tdt, device="cuda") for A, w in zip(mats, widths)]
        best = None
        for C in Cs:
            for sigma in sigmas:
                if 1 < sigma < C:
                    continue
                S = [sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=dtype) for A in mats]
                for pol in LANE_POLICIES:
                    cpl = [_policy_cpl(int(w), xs, pol) for w in widths]
                    b = sellcs.Batch(S, widths, cols_per_lane=cpl, vec_dtype=vec_dtype)
                    b.bind(xv, yv)
                    us = _time_batch(b, reps)
                    b.close()
                    if best is None or us < best[0]:
                        best = (us, C, sigma, pol)
                for m in S:
                    m.close()
        us, C, sigma, pol = best
        cache[key] = {"C": C, "sigma": sigma, "policy": pol, "us": round(us, 2)}
        _store_cache(cache_path, cache)
    e = cache[key]
    xs = 4 if vec_dtype == "f32" else 8
    return [{"C": e["C"], "sigma": e["sigma"], "cpl": _policy_cpl(int(w), xs, e["policy"]), "us": e["us"]}
            for w in widths]


def _load_cache(cache_path):
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def _store_cache(cache_path, cache):
    if not cache_path:
        return
    os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
    tmp = cache_path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=0, sort_keys=True)
    os.replace(tmp, cache_path)


def tune_batch(mats, widths, dtype: str = "f32", vec_dtype: str = "f32", cache_path: str | None = DEFAULT_CACHE,
               reps: int = 20, Cs=C_CANDIDATES, sigmas=SIGMA_CANDIDATES):
    """Per-matrix {C, sigma, cpl, us}, each matrix timed on its own; cached by
    structural signature."""
    cache = _load_cache(cache_path)
    out = []
    dirty = False
    for A, w in zip(mats, widths):
        key = signature(A, w, dtype)
        if key not in cache:
            cache[key] = tune_matrix(A, int(w), dtype, vec_dtype, reps, Cs, sigmas)
            dirty = True
        out.append(cache[key])
    if dirty:
        _store_cache(cache_path, cache)
    return out


SPMV_C_CANDIDATES = (4, 8, 16, 32)
SPMV_ORDERS = ("front", "ranges")


def tune_spmv(A, w: int, dtype: str = "f64", vec_dtype: str = "f64", with_transpose: bool = False,
              cache_path: str | None = DEFAULT_CACHE, reps: int = 20, Cs=SPMV_C_CANDIDATES, sigmas=None,
              orders=SPMV_ORDERS) -> dict:
    """{C, sigma, order, us} for y = A x through sp_spmv at block width w (and,
    with ``with_transpose``, the adjoint sp_spmv_adjoint as well: the objective
    is then the forward plus the backward time).  sigma candidates default to
    1, 256 and the whole matrix."""
    import torch
    key = f"spmv:{signature(A, w, dtype)}:{vec_dtype}:{int(with_transpose)}"
    cache = _load_cache(cache_path)
    if key not in cache:
        if sigmas is None:
            sigmas = tuple(sorted({1, 256, max(1, int(A.nrows))}))
        tdt = torch.float32 if vec_dtype == "f32" else torch.float64
        x = torch.rand(A.ncols, w, dtype=tdt, device="cuda")
        y = torch.empty(A.nrows, w, dtype=tdt, device="cuda")
        g = torch.rand(A.nrows, w, dtype=tdt, device="cuda") if with_transpose else None
        dx = torch.empty_like(x) if with_transpose else None
        dv = torch.empty(A.nnz, dtype=tdt, device="cuda") if with_transpose else None
        best = None
        for C in Cs:
            for sigma in sigmas:
                if 1 < sigma < C:
                    continue
                for order in orders:
                    m = sellcs.SellMatrix(A, C=C, sigma=sigma, dtype=dtype, with_transpose=with_transpose,
                                          order=order)

                    def step():
                        sellcs.spmv(m, x, y)
                        if with_transpose:
                            sellcs.spmv_adjoint(m, g, x=x, dx=dx, dvals=dv)

                    for _ in range(3):
                        step()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    for _ in range(reps):
                        step()
                    e1.record()
                    torch.cuda.synchronize()
                    us = e0.elapsed_time(e1) * 1e3 / reps
                    m.close()
                    if best is None or us < best["us"]:
                        best = {"C": C, "sigma": int(sigma), "order": order, "us": round(us, 2)}
        cache[key] = best
        _store_cache(cache_path, cache)
    return dict(cache[key])
