#!/usr/bin/env python
"""Benchmark of the SELL-C-sigma augmented SpMMV on one GB300 (or N replicas).

Headline workload (the augmented product on an irregular matrix):
  N = 2^21 rows, row lengths uniform in [4, 64], 90 % of columns within +-4096
  of the diagonal and 10 % uniform, float64 values uniform(-1, 1); SELL-32-256;
  y = 0.5 (A - 0.1 I) x + 1.0 y with <x,y>, <y,y> and z = 0.9 z + 0.1 y.
One step = one sp_spmv call (a single kernel launch: product, epilogue, dots
and chain fused).  Inputs (about 0.96 GB) are larger than the 129 MB L2, so no
flush is needed between steps.

metric: effective HBM bandwidth = algorithmic bytes per call / time, where the
algorithmic bytes count every real nonzero's value and index once, x once,
y read (beta) and written, z read and written, and the per-row/per-chunk
metadata (padding is excluded).

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU
oracle instead (the paper-derived reference program), on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="irregular_band_augmented", N=1 << 21, rowlen="U[4,64]", band=4096, p_band=0.9,
                values="f64 U(-1,1)", C=32, sigma=256, w=1, alpha=0.5, gamma=0.1, beta=1.0, delta=0.9, eta=0.1,
                dots="xy,yy", chain=True)


def algorithmic_bytes(nnz, nrows, ncols, nchunks, nslots, w, sv, sx, axpby, chain, permuted):
    """Bytes a perfect-cache run must move per call (padding excluded)."""
    b = nnz * (sv + 4)                    # values + int32 column indices
    b += ncols * w * sx                   # x, once
    b += nrows * w * sx * (1 + int(axpby))  # y written (and read for beta)
    b += int(chain) * 2 * nrows * w * sx  # z read + written
    b += nchunks * 8 + nslots * 4         # chunk offsets + per-slot row lengths
    b += int(permuted) * nslots * 4       # permutation
    return int(b)


METRIC = "SpMMV effective HBM GB/s (augmented SELL-32-256, f64, irregular N=2^21)"
DATA = "synthetic (seeded irregular band matrix standing in for the paper's SuiteSparse inputs)"
FP64_NOMINAL_TFLOPS = 1.25  # nominal dense float64 rate of a GB300 (context only)


def measured_fp64_rate():
    """Float64 fused multiply-add rate of this GPU (the library's DFMA-chain
    micro-benchmark, sp_device_fp64_rate), with the SM clocks sampled while it
    ran."""
    from paper_1507_08101_gb300 import sellcs
    import torch
    with ClockSampler(torch.cuda.current_device()) as clk:
        best = 0.0
        for _ in range(3):
            t, ms = sellcs.device_fp64_rate()
            best = max(best, t)
    c = clk.summary()
    out = {"tflops": round(best, 4), "launch_ms": round(ms, 3), "clocks": c,
           "method": "sp_device_fp64_rate: 2048 threads per SM x 16 independent fma chains x 8192 steps, "
                     "best of 3 calls (each the best of 3 event-timed launches)"}
    if c and c.get("sm_mhz"):
        out["per_sm_per_cycle_fma"] = round(best * 1e12 / 2 / (c["sm_mhz"] * 1e6) / torch.cuda.get_device_properties(
            torch.cuda.current_device()).multi_processor_count, 3)
    return out


def fp64_derived_peak(meas):
    """Float64 peak from the unit count and the clock: 2 fused multiply-adds
    per SM and cycle (one float64 warp instruction about every 16 SM cycles)
    x SMs x the maximum SM clock x 2 flops.  The DFMA-chain micro-benchmark
    (sp_device_fp64_rate) reaches about 0.85 of it, below what the float64
    tall-skinny product sustains (0.95), so it is reported beside the derived
    figure rather than used as the ceiling."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (meas.get("clocks") or {}).get("sm_max_mhz") or 2070.0
    peak = 2 * 2 * sms * mhz * 1e6 / 1e12
    kind = f"derived: 2 float64 fma per SM per cycle x {sms} SMs x {mhz:.0f} MHz x 2 flops"
    if meas.get("tflops"):
        kind += f"; measured DFMA-chain rate {meas['tflops']} TFLOP/s beside it"
    return round(peak, 4), kind


def fp64_flops(nnz, nrows, w, shift, scale, axpby, ndots, chain):
    """float64 flops of one call: the row sums (2 per nonzero and column) and
    the epilogue per row and column (fma = 2, mul = 1)."""
    per = 2 * int(shift) + int(scale) + 2 * int(axpby) + 2 * ndots + 3 * int(chain)
    return 2 * nnz * w + per * nrows * w


def max_over_ranks(x: float) -> float:
    """Largest value of x over the ranks of the default process group (x itself
    when the run is not distributed): the job's time is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Units per second of the whole job: every rank (an independent replica)
    processes units_per_rank in the slowest rank's time ms_max."""
    return units_per_rank * world / (ms_max * 1e-3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for fn in ("spmv_kernel.cuh", "spmv_launch.cuh"):
        with open(os.path.join(ROOT, "paper_1507_08101_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(name):
    """Per-launch DRAM bytes from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+kernel_src_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload():
    from workloads import generators as gen
    A, x, y0, z0 = gen.workload_irregular(WORKLOAD["N"])
    return A, x, y0, z0


# ------------------------------------------------------------------ our arm


def run_ours(args, rank, world):
    import torch
    from paper_1507_08101_gb300 import sellcs
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    A, X, Y0, Z0 = make_workload()
    W = WORKLOAD
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # one small build first, so the timed build excludes one-time module loading
        from workloads import generators as _gen
        sellcs.SellMatrix(_gen.laplace2d(8, 0.0), C=W["C"], sigma=W["sigma"], dtype="f64").close()
        torch.cuda.synchronize()
        t0 = time.time()
        mat = sellcs.SellMatrix(A, C=W["C"], sigma=W["sigma"], dtype="f64")
        torch.cuda.synchronize()
        setup_s = time.time() - t0
        info = mat.info()
        x = torch.from_numpy(X).to(dev)
        y = torch.from_numpy(Y0).to(dev)
        z = torch.from_numpy(Z0).to(dev)
        dot = torch.zeros(3, dtype=torch.float64, device=dev)
        nbytes = algorithmic_bytes(A.nnz, A.nrows, A.ncols, info["nchunks"], info["nchunks"] * info["C"], 1, 8, 8,
                                   True, True, W["sigma"] > 1)
        hx, hy, hz = sellcs.sp_dense_view(x), sellcs.sp_dense_view(y), sellcs.sp_dense_view(z)
        import ctypes as ct
        opts, keep = sellcs.make_opts(1, alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], dot_xy=True,
                                      dot_yy=True, z_handle=hz, delta=W["delta"], eta=W["eta"],
                                      dot_ptr=ct.c_void_p(dot.data_ptr()))
        L = sellcs.lib()
        sp = ct.c_void_p(stream.cuda_stream)

        def step():
            rc = L.sp_spmv(hy, mat.handle, hx, ct.byref(opts), sp)
            if rc:
                sellcs.check(rc, "sp_spmv")

        for _ in range(args.warmup):
            step()
        stream.synchronize()
        # the values of y and z drift over repeated steps (beta = 1): harmless for timing
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(dev.index) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                step()
            ev1.record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(ev0.elapsed_time(ev1))
        ms_step = ms / args.steps

        # e2e: the library's host-buffer entry point (sp_spmv_host on a host plan):
        # every step copies x, y, z in from page-locked host memory and y, z and
        # the dots back, inside the timed region; consecutive steps overlap their
        # copies with the product of the step between them
        hx_h = torch.from_numpy(X).pin_memory()
        hy_h = torch.from_numpy(Y0).pin_memory()
        hz_h = torch.from_numpy(Z0).pin_memory()
        oy = torch.empty_like(hy_h).pin_memory()
        oz = torch.empty_like(hz_h).pin_memory()
        od = torch.empty(3, dtype=torch.float64).pin_memory()
        plan = sellcs.HostPlan(mat, 1, "f64")
        kw = dict(alpha=WORKLOAD["alpha"], gamma=WORKLOAD["gamma"], beta=WORKLOAD["beta"], dot_xy=True, dot_yy=True,
                  delta=WORKLOAD["delta"], eta=WORKLOAD["eta"])

        def e2e_step():
            plan.spmv(hx_h, oy, y_in=hy_h, z_in=hz_h, z_out=oz, dot=od, **kw)

        for _ in range(max(3, args.warmup)):
            e2e_step()
        plan.sync()
        e2e_steps = max(3, min(args.steps, 200))
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        plan.sync()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3) / e2e_steps
        plan.close()
        h2d = X.nbytes + Y0.nbytes + Z0.nbytes
        d2h = Y0.nbytes + Z0.nbytes + 2 * 8

        # per-call rates in the manner of the paper's spmvbench (Sec.
        # "Heterogeneous execution"): P_max = the best of 100 calls, P_skip10 =
        # the mean rate of all but the first ten; each call between its own events
        calls = 100
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
        torch.cuda.synchronize()
        for a, b in evs:
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        per_ms = np.array([a.elapsed_time(b) for a, b in evs])
        gf = 2.0 * A.nnz / (per_ms * 1e-3) / 1e9
        gb = nbytes / (per_ms * 1e-3) / 1e9
        spmvbench = {"calls": calls, "P_max_GFs": round(float(gf.max()), 2),
                     "P_skip10_GFs": round(float(gf[10:].mean()), 2), "P_max_GBs": round(float(gb.max()), 1),
                     "P_skip10_GBs": round(float(gb[10:].mean()), 1),
                     "note": "GF/s = 2 nnz / call time, as the paper's spmvbench; GB/s = algorithmic bytes / call time"}

        # value-only update (Sec. "Sparse matrix storage": a later construction
        # with the same pattern only updates the values), values already on the
        # device, against the product time
        vdev = torch.from_numpy(A.val).to(dev)
        mat.update_values(vdev, stream)
        torch.cuda.synchronize()
        upd_ms = _events_time(lambda: mat.update_values(vdev, stream), 10, stream)
        del vdev
        for h in (hx, hy, hz):
            sellcs.sp_dense_destroy(h)

    gbs = nbytes / (ms_step * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    flops = fp64_flops(A.nnz, A.nrows, 1, True, True, True, 2, True)
    tflops = flops / (ms_step * 1e-3) / 1e12
    # the DFMA-chain probe runs after the timed region; --no-fp64-probe leaves
    # it out (a launch list of the product path alone), the derived peak stays
    fp64 = measured_fp64_rate() if not args.no_fp64_probe else {}
    fp64_peak, fp64_kind = fp64_derived_peak(fp64)
    hbm = {"bound": "hbm", "achieved": round(gbs, 2), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
           "peak_kind": f"{peak_kind} copy bandwidth (burst)",
           "traffic": recorded_traffic("k_spmmv_irregular_augmented.md"),
           "kernel": "k_spmmv<double,double,1,VEC,DOTS,!MT>",
           "algorithmic_bytes_per_launch": nbytes}
    alu = {"bound": "alu", "achieved": round(tflops, 4), "peak": fp64_peak, "unit": "TFLOP/s",
           "frac": round(tflops / fp64_peak, 4),
           "peak_kind": fp64_kind, "fp64_flops_per_launch": flops, "fp64_rate_measurement": fp64}
    # the binding resource is the one closest to its ceiling; the other is reported beside it
    roof = dict(alu if alu["frac"] > hbm["frac"] else hbm)
    roof["other"] = hbm if roof["bound"] == "alu" else alu
    result = {
        "metric": METRIC,
        "value": round(whole_job_rate(nbytes, ms_step, world) / 1e9, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": DATA,
        "config": workload_config(A, nbytes, world),
        "roofline": roof,
        "e2e": {"value": round(whole_job_rate(nbytes, e2e_ms, world) / 1e9, 2), "unit": "GB/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 4),
                "api": "sp_spmv_host on a host plan (pinned buffers, copies of consecutive steps overlapped)",
                "steps": e2e_steps},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "setup": {"nstored": info["nstored"], "sell_build_s": round(setup_s, 4), "in_spmv_calls": round(setup_s / (ms_step * 1e-3), 1),
                  "update_values_device_ms": round(upd_ms, 4),
                  "update_values_in_spmv_calls": round(upd_ms / ms_step, 2)},
        "spmvbench": spmvbench,
    }
    return result, (A, X, Y0, Z0)


# ------------------------------------------------------------------ secondary workloads


def _events_time(fn, reps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps  # ms


def secondary_laplace(peak, sizes=(32, 256)):
    """Laplacian 32^3 (SELL-32-1, plain y = A x, f64): cold (L2 flushed before
    each launch) and warm (CUDA graph of 1000 back-to-back launches), plus the
    same stencil at 256^3 as the HBM-bound companion."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    from workloads import generators as gen
    out = {}
    for n in sizes:
        A = gen.laplace3d(n)
        m = sellcs.SellMatrix(A, C=32, sigma=1)
        inf = m.info()
        x = torch.from_numpy(gen.block_vector(A.nrows, 1, gen.BASE_SEED + 1)[:, 0]).cuda()
        y = torch.zeros_like(x)
        nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * 32, 1, 8, 8, False, False,
                               False)
        stream = torch.cuda.Stream()
        hx, hy = sellcs.sp_dense_view(x), sellcs.sp_dense_view(y)
        import ctypes as ct
        o, _ = sellcs.make_opts(1)
        L = sellcs.lib()
        sp = ct.c_void_p(stream.cuda_stream)

        def call():
            L.sp_spmv(hy, m.handle, hx, ct.byref(o), sp)

        with torch.cuda.stream(stream):
            for _ in range(5):
                call()
            torch.cuda.synchronize()
            flush = torch.empty(2 * 129 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
            cold = []
            for _ in range(20):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                torch.cuda.synchronize()
                cold.append(e0.elapsed_time(e1))
            del flush
            cold_ms = statistics.median(cold)
            g = torch.cuda.CUDAGraph()
            R = 1000 if n == 32 else 20
            with torch.cuda.graph(g, stream=stream):
                for _ in range(R):
                    call()
            g.replay()
            torch.cuda.synchronize()
            warm_ms = _events_time(g.replay, 5, stream) / R
        sellcs.sp_dense_destroy(hx)
        sellcs.sp_dense_destroy(hy)
        out[f"laplace{n}"] = {"nnz": A.nnz, "bytes_per_call": nb,
                              "cold_us": round(cold_ms * 1e3, 2), "cold_GBs": round(nb / cold_ms / 1e6, 1),
                              "warm_graph_us": round(warm_ms * 1e3, 3), "warm_graph_GBs": round(nb / warm_ms / 1e6, 1),
                              "warm_frac_of_peak": round(nb / warm_ms / 1e6 / peak, 4)}
        del m, x, y
    if "laplace32" in out:
        out["laplace32"]["note"] = ("3.2 MB working set: the warm number is served from L2 and is not an HBM figure; "
                                    "the cold number is dominated by launch and ramp latency")
    return out


def _row_sample_csr(A, rows):
    from workloads.generators import CSR
    lens = A.rowptr[rows + 1] - A.rowptr[rows]
    rp = np.zeros(rows.size + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    idx = np.concatenate([np.arange(A.rowptr[r], A.rowptr[r + 1]) for r in rows])
    return CSR(rows.size, A.ncols, rp, A.col[idx], A.val[idx])


ANDERSON_PAIRS = [("f64", "f64"), ("f32", "f64"), ("bf16", "f64"), ("f32", "f32"), ("bf16", "f32")]


def secondary_anderson(peak, pairs=None):
    """Anderson 128^3, width-16 Chebyshev step (alpha = 2/a, beta = -1) in each
    precision pair (values, vectors): GB/s, speedup over f64, max error on 2048
    sampled rows against the f64 oracle (relative to max |y|).  ``pairs``
    restricts the run to some of the pairs (the speed-up is then relative to
    the first pair run)."""
    import ctypes as ct
    import torch
    import oracle
    from paper_1507_08101_gb300 import sellcs
    from workloads import generators as gen
    A, X = gen.workload_anderson()
    a = 1.01 * (6 + 8.25)
    rows = np.sort(np.random.default_rng(0).choice(A.nrows, 2048, replace=False))
    sub = _row_sample_csr(A, rows)
    Y0 = gen.block_vector(A.nrows, 16, gen.BASE_SEED + 2, tag=77)
    yref = oracle.spmmv(sub, X, alpha=2 / a, beta=-1.0, y0=Y0[rows])[0]
    out = {}
    base = None
    for vdt, xdt in (pairs or ANDERSON_PAIRS):
        m = sellcs.SellMatrix(A, C=32, sigma=1, dtype=vdt)
        inf = m.info()
        tdt = torch.float64 if xdt == "f64" else torch.float32
        x = torch.from_numpy(X).to("cuda", tdt)
        y0 = torch.from_numpy(Y0).to("cuda", tdt)
        y = y0.clone()
        hx, hy = sellcs.sp_dense_view(x), sellcs.sp_dense_view(y)
        o, _ = sellcs.make_opts(16, alpha=2 / a, beta=-1.0)
        L = sellcs.lib()
        stream = torch.cuda.current_stream()
        sp = ct.c_void_p(stream.cuda_stream)
        L.sp_spmv(hy, m.handle, hx, ct.byref(o), sp)
        torch.cuda.synchronize()
        err = float(np.abs(y.double().cpu().numpy()[rows] - yref).max() / np.abs(yref).max())
        for _ in range(3):
            L.sp_spmv(hy, m.handle, hx, ct.byref(o), sp)
        ms = _events_time(lambda: L.sp_spmv(hy, m.handle, hx, ct.byref(o), sp), 30, stream)
        sv = {"f64": 8, "f32": 4, "bf16": 2}[vdt]
        sx = 8 if xdt == "f64" else 4
        nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * 32, 16, sv, sx, True,
                               False, False)
        if base is None:
            base = ms
        out[f"{vdt}_vals_{xdt}_vecs"] = {"us": round(ms * 1e3, 1), "GBs": round(nb / ms / 1e6, 1),
                                         "frac_of_peak": round(nb / ms / 1e6 / peak, 4),
                                         "speedup_vs_f64": round(base / ms, 3), "max_rel_err_vs_f64_oracle": err,
                                         "bytes_per_call": nb}
        sellcs.sp_dense_destroy(hx)
        sellcs.sp_dense_destroy(hy)
        del m, x, y, y0
    return out


def secondary_powerlaw(peak, fixed=None):
    """Power-law N = 2^20, f32, width 4: forward product and backward
    (A^T g through the transposed matrix + sampled dvals).  ``fixed`` =
    (C, sigma, order) skips the autotuner (a profiler run, whose timings would
    mislead the tuner)."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    from workloads import generators as gen
    from paper_1507_08101_gb300 import autotune
    A, X, G = gen.workload_powerlaw()
    t0 = time.perf_counter()
    if fixed:
        tuned = {"C": int(fixed[0]), "sigma": int(fixed[1]), "order": fixed[2]}
    else:
        tuned = autotune.tune_spmv(A, 4, "f32", "f32", with_transpose=True, cache_path=None)
    tune_s = time.perf_counter() - t0
    m = sellcs.SellMatrix(A, C=tuned["C"], sigma=tuned["sigma"], dtype="f32", with_transpose=True,
                          order=tuned["order"])
    inf = m.info()
    x = torch.from_numpy(X).to("cuda", torch.float32)
    g = torch.from_numpy(G).to("cuda", torch.float32)
    y = torch.empty_like(x)
    dx = torch.empty_like(x)
    dv = torch.empty(A.nnz, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        sellcs.spmv(m, x, y)
        sellcs.spmv_adjoint(m, g, x=x, dx=dx, dvals=dv)
    fwd = _events_time(lambda: sellcs.spmv(m, x, y), 50, stream)
    bwd = _events_time(lambda: sellcs.spmv_adjoint(m, g, x=x, dx=dx, dvals=dv), 50, stream)
    C = tuned["C"]
    nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * C, 4, 4, 4, False, False,
                           tuned["sigma"] > 1)
    # backward: A^T product (same byte count) + sampled: col index + dvals write per nonzero, g and x once
    nb_bwd = nb + A.nnz * (4 + 4) + 2 * A.nrows * 4 * 4 + inf["nchunks"] * C * 8
    return {"nnz": A.nnz, "tuned": {k: tuned[k] for k in ("C", "sigma", "order")}, "autotune_s": round(tune_s, 2),
            "nstored": inf["nstored"], "fwd_us": round(fwd * 1e3, 1), "fwd_GBs": round(nb / fwd / 1e6, 1),
            "bwd_us": round(bwd * 1e3, 1), "bwd_GBs": round(nb_bwd / bwd / 1e6, 1)}


def secondary_permuted(peak):
    """The bench product (irregular N = 2^21, SELL-32-256, augmented) with the
    vectors in SELL row order (SP_MAT_PERMUTED_SPACE): same algorithmic bytes,
    x_i, y and z accessed at consecutive rows of a chunk."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    A, X, Y0, Z0 = make_workload()
    W = WORKLOAD
    out = {}
    for name, perm in (("user_order", False), ("sell_order", True)):
        m = sellcs.SellMatrix(A, C=W["C"], sigma=W["sigma"], dtype="f64", permuted=perm)
        inf = m.info()
        x, y, z = (torch.from_numpy(v).cuda() for v in (X, Y0, Z0))
        if perm:
            xp, yp, zp = torch.empty_like(x), torch.empty_like(y), torch.empty_like(z)
            for src, dst in ((x, xp), (y, yp), (z, zp)):
                sellcs.mat_permute(m, dst, src, True)
            x, y, z = xp, yp, zp
        dot = torch.zeros(3, dtype=torch.float64, device="cuda")
        kw = dict(alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], dot_xy=True, dot_yy=True, z=z,
                  delta=W["delta"], eta=W["eta"], dot=dot)
        for _ in range(5):
            sellcs.spmv(m, x, y, **kw)
        torch.cuda.synchronize()
        ms = _events_time(lambda: sellcs.spmv(m, x, y, **kw), 200, torch.cuda.current_stream())
        nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * W["C"], 1, 8, 8, True, True,
                               W["sigma"] > 1)
        out[name] = {"us": round(ms * 1e3, 1), "GBs": round(nb / ms / 1e6, 1), "frac_of_peak": round(nb / ms / 1e6 / peak, 4)}
        m.close()
    return out


def secondary_vty(peak):
    """The bench product (irregular N = 2^21, SELL-32-256, f64, w = 1,
    shift/scale/beta and the chain) fused with C = V^T y for a block V of m
    columns (sp_spmv_vty), against the same product followed by a separate
    tall-skinny pass (sp_spmv, then sp_tsmttsm over V and y).  The fused form
    saves one read of y; both read V once."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    A, X, Y0, Z0 = make_workload()
    W = WORKLOAD
    m = sellcs.SellMatrix(A, C=W["C"], sigma=W["sigma"], dtype="f64")
    inf = m.info()
    x, y, z = (torch.from_numpy(v).cuda() for v in (X, Y0, Z0))
    kw = dict(alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], z=z, delta=W["delta"], eta=W["eta"])
    nb_prod = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * W["C"], 1, 8, 8, True, True,
                                W["sigma"] > 1)
    stream = torch.cuda.current_stream()
    out = {}
    for mm in (1, 4, 8):
        g = torch.Generator(device="cuda")
        g.manual_seed(1000 + mm)
        V = torch.rand(A.nrows, mm, dtype=torch.float64, device="cuda", generator=g) - 0.5
        Cf = torch.empty(mm, 1, dtype=torch.float64, device="cuda")
        Cu = torch.empty(mm, 1, dtype=torch.float64, device="cuda")
        y2 = y.view(-1, 1)

        def fused():
            sellcs.spmv_vty(m, x, y, V, Cf, **kw)

        def unfused():
            sellcs.spmv(m, x, y, **kw)
            sellcs.tsmttsm(Cu, V, y2)

        for _ in range(5):
            fused()
            unfused()
        torch.cuda.synchronize()
        tf = _events_time(fused, 100, stream)
        tu = _events_time(unfused, 100, stream)
        nb_f = nb_prod + A.nrows * mm * 8
        nb_u = nb_prod + A.nrows * (mm + 1) * 8
        out[f"m{mm}"] = {"fused_us": round(tf * 1e3, 1), "fused_GBs": round(nb_f / tf / 1e6, 1),
                         "unfused_us": round(tu * 1e3, 1), "unfused_GBs_of_its_bytes": round(nb_u / tu / 1e6, 1),
                         "speedup_fused": round(tu / tf, 3)}
    m.close()
    return out


def secondary_dist(peak):
    """The row-partitioned product of the bench workload with P parts on this
    one GPU (dist.LocalWorld: every part's halo pack, the halo copies and every
    part's product, one after another on one stream), in the overlapped
    two-pass form and the one-pass form, against the single product.  On one
    GPU nothing overlaps: this measures what the split itself costs (the
    two-pass form reads and writes y twice, as the paper notes for its
    overlapped modes) and how large the halo is."""
    import torch
    from paper_1507_08101_gb300 import dist, sellcs
    A, X, Y0, Z0 = make_workload()
    W = WORKLOAD
    nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, (A.nrows + 31) // 32, ((A.nrows + 31) // 32) * 32, 1, 8, 8,
                           True, True, True)
    kw = dict(alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], dot_xy=True, dot_yy=True, delta=W["delta"],
              eta=W["eta"])
    out = {}
    m = sellcs.SellMatrix(A, C=W["C"], sigma=W["sigma"], dtype="f64")
    x, y, z = (torch.from_numpy(v).cuda() for v in (X, Y0, Z0))
    for _ in range(3):
        sellcs.spmv(m, x, y, z=z, **kw)
    torch.cuda.synchronize()
    ms = _events_time(lambda: sellcs.spmv(m, x, y, z=z, **kw), 50, torch.cuda.current_stream())
    out["single"] = {"us": round(ms * 1e3, 1), "GBs": round(nb / ms / 1e6, 1)}
    m.close()
    del x, y, z
    for P in (2, 4):
        for mode in ("overlap", "no_overlap"):
            world = dist.LocalWorld(A, P, C=W["C"], sigma=W["sigma"], mode=mode)
            xs = world.scatter(torch.from_numpy(X))
            ys = [torch.from_numpy(Y0[world.bounds[r]:world.bounds[r + 1]]).cuda() for r in range(P)]
            zs = [torch.from_numpy(Z0[world.bounds[r]:world.bounds[r + 1]]).cuda() for r in range(P)]
            for _ in range(3):
                world.spmv(xs, ys, zs, **kw)
            torch.cuda.synchronize()
            ms = _events_time(lambda: world.spmv(xs, ys, zs, **kw), 20, torch.cuda.current_stream())
            halo = sum(p.info()["nhalo"] for p in world.plans)
            rem = sum(p.info()["nnz_remote"] for p in world.plans)
            out[f"P{P}_{mode}"] = {"us": round(ms * 1e3, 1), "GBs_of_single_bytes": round(nb / ms / 1e6, 1),
                                   "halo_rows": int(halo), "remote_nnz_frac": round(rem / A.nnz, 4)}
            for mm in world.mats:
                mm.close()
            del world, xs, ys, zs
    return out


def secondary_tsm(peak, dtypes=("f64", "f32")):
    """Tall and skinny kernels on n = 2^22 rows, m = k = 16: V^T W (plain and
    Kahan) and V X.  Bytes: V and W read once (tsmttsm); V read, W written
    (tsmm, beta = 0); flops 2 n m k."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    n, m, k = 1 << 22, 16, 16
    out = {"n": n, "m": m, "k": k}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        if dt not in dtypes:
            continue
        g = torch.Generator(device="cuda").manual_seed(5)
        V = torch.rand(n, m, dtype=tdt, device="cuda", generator=g)
        W = torch.rand(n, k, dtype=tdt, device="cuda", generator=g)
        X = torch.zeros(m, k, dtype=tdt, device="cuda")
        S = torch.rand(m, k, dtype=tdt, device="cuda", generator=g)
        es = V.element_size()
        res = {}
        for name, fn, nbytes in (
                ("tsmttsm", lambda: sellcs.tsmttsm(X, V, W, 1.0, 0.0, False), n * (m + k) * es),
                ("tsmttsm_kahan", lambda: sellcs.tsmttsm(X, V, W, 1.0, 0.0, True), n * (m + k) * es),
                ("tsmm", lambda: sellcs.tsmm(W, V, S, 1.0, 0.0), n * (m + k) * es)):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            ms = _events_time(fn, 20, torch.cuda.current_stream())
            res[name] = {"us": round(ms * 1e3, 1), "GBs": round(nbytes / ms / 1e6, 1),
                         "TFLOPs": round(2.0 * n * m * k / ms / 1e9, 3)}
        out[dt] = res
    return out


def secondary_kpm(peak):
    """KPM moments on the Anderson 128^3 matrix with a width-16 block (the
    solver the fused product serves): 128 moments from 64 fused products
    (sp_kpm_moments), against the same Chebyshev loop with the products
    unfused (sp_spmv without dots, then the two inner products as separate
    passes over the block vectors: torch reductions, a comparison only)."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    from workloads import generators as gen
    A, X = gen.workload_anderson()
    a = 1.01 * (6 + 8.25)
    nmom = 128
    out = {"nmom": nmom, "w": 16}
    for vdt, xdt in (("f64", "f64"), ("f32", "f32")):
        tdt = torch.float64 if xdt == "f64" else torch.float32
        m = sellcs.SellMatrix(A, C=32, sigma=1, dtype=vdt)
        x = torch.from_numpy(X).to("cuda", tdt)
        sellcs.kpm_moments(m, x, nmom, a, 0.0)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            mu = sellcs.kpm_moments(m, x, nmom, a, 0.0)
        fused = (time.perf_counter() - t0) / reps

        def unfused():
            u = x.clone()
            v = torch.empty_like(u)
            mu0 = (u * u).sum(0)
            sellcs.spmv(m, u, v, alpha=1 / a)
            mus = [mu0, (u * v).sum(0)]
            for n in range(1, nmom // 2):
                sellcs.spmv(m, v, u, alpha=2 / a, beta=-1.0)
                mus.append(2 * (v * v).sum(0) - mu0)  # mu_{2n}
                mus.append(2 * (u * v).sum(0) - mus[1])  # mu_{2n+1}
                u, v = v, u
            return torch.stack(mus[:nmom]).cpu()

        unfused()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            mu_u = unfused()
        torch.cuda.synchronize()
        unf = (time.perf_counter() - t0) / reps
        rel = float(np.max(np.abs(mu - mu_u.double().numpy()) / np.abs(mu[0])))
        res = {"fused_ms": round(fused * 1e3, 2), "per_product_us": round(fused / (nmom // 2) * 1e6, 1),
               "unfused_ms": round(unf * 1e3, 2), "speedup_fused": round(unf / fused, 2),
               "max_rel_diff_fused_vs_unfused": rel}
        # blocking (Sec. "Kernel fusion": blocking and fusion together): the
        # same 16 starts run one vector at a time, fused and unfused
        cols = [x[:, k:k + 1].contiguous() for k in range(x.shape[1])]
        t0 = time.perf_counter()
        for c in cols:
            sellcs.kpm_moments(m, c, nmom, a, 0.0)
        torch.cuda.synchronize()
        f1 = time.perf_counter() - t0
        x_all = x
        t0 = time.perf_counter()
        for c in cols:
            x = c
            unfused()
        torch.cuda.synchronize()
        u1 = time.perf_counter() - t0
        x = x_all
        res.update({"w1x16_fused_ms": round(f1 * 1e3, 2), "w1x16_unfused_ms": round(u1 * 1e3, 2),
                    "speedup_blocking": round(f1 / fused, 2), "speedup_blocking_and_fusion": round(u1 / fused, 2)})
        out[f"{vdt}_vals_{xdt}_vecs"] = res
        m.close()
    return out


def secondary_layout(peak):
    """Row-major (interleaved) against column-major block vectors (Sec. "Block
    vectors"): the Anderson 128^3 Chebyshev step at width 16 (and 4) with x and
    y in either layout, same algorithmic bytes."""
    import torch
    from paper_1507_08101_gb300 import sellcs
    from workloads import generators as gen
    A, X = gen.workload_anderson()
    a = 1.01 * (6 + 8.25)
    out = {}
    for vdt, xdt in (("f64", "f64"), ("f32", "f32")):
        tdt = torch.float64 if xdt == "f64" else torch.float32
        m = sellcs.SellMatrix(A, C=32, sigma=1, dtype=vdt)
        inf = m.info()
        for w in (16, 4):
            res = {}
            for lay in ("row", "col"):
                xr = torch.from_numpy(np.ascontiguousarray(X[:, :w])).to("cuda", tdt)
                if lay == "row":
                    x, y = xr, torch.zeros_like(xr)
                    L = sellcs.SP_ROW_MAJOR
                else:
                    x = xr.t().contiguous().t()  # (N, w) with unit row stride
                    y = torch.zeros_like(xr).t().contiguous().t()
                    L = sellcs.SP_COL_MAJOR
                for _ in range(3):
                    sellcs.spmv(m, x, y, alpha=2 / a, beta=-1.0, layout=L)
                torch.cuda.synchronize()
                ms = _events_time(lambda: sellcs.spmv(m, x, y, alpha=2 / a, beta=-1.0, layout=L), 20,
                                  torch.cuda.current_stream())
                sv = 8 if vdt == "f64" else 4
                nb = algorithmic_bytes(A.nnz, A.nrows, A.ncols, inf["nchunks"], inf["nchunks"] * 32, w, sv, sv, True,
                                       False, False)
                res[lay] = {"us": round(ms * 1e3, 1), "GBs": round(nb / ms / 1e6, 1)}
            res["row_over_col_speedup"] = round(res["col"]["us"] / res["row"]["us"], 3)
            out[f"{vdt}_{xdt}_w{w}"] = res
        m.close()
    return out


def secondary_cg_batch(peak):
    """64 SPD systems L_2D(s) + 0.01 I, s in [64, 512], widths 1..8.
    (a) one persistent batched f32 SpMMV launch vs one batched f64 launch vs 64
    separate plain f64 sp_spmv launches; (b) mixed-precision CG time to
    ||b - Ax|| <= 1e-10 ||b|| (f32 inner, graph-captured) vs the same driver
    with a f64 inner solve.  C, sigma and lanes per row from the autotuner."""
    import time as _t
    import torch
    from paper_1507_08101_gb300 import autotune, sellcs
    from workloads import generators as gen
    batch = gen.workload_cg_batch()
    mats = [A for A, _ in batch]
    Bs = [B for _, B in batch]
    widths = [B.shape[1] for B in Bs]
    t0 = _t.time()
    cfg = autotune.tune_batch_joint(mats, widths, dtype="f32", vec_dtype="f32",
                              cache_path=os.path.join(ROOT, "_autotune_cache.json"))
    tune_s = _t.time() - t0
    S64 = [sellcs.SellMatrix(A, C=c["C"], sigma=c["sigma"], dtype="f64") for A, c in zip(mats, cfg)]
    S32 = [s.clone("f32") for s in S64]
    cpl32 = [c["cpl"] for c in cfg]
    xs32 = [torch.rand(A.nrows, w, dtype=torch.float32, device="cuda") for A, w in zip(mats, widths)]
    ys32 = [torch.empty_like(v) for v in xs32]
    xs64 = [v.double() for v in xs32]
    ys64 = [torch.empty_like(v) for v in xs64]
    b32 = sellcs.Batch(S32, widths, cols_per_lane=cpl32, vec_dtype="f32")
    b32.bind(xs32, ys32)
    b64 = sellcs.Batch(S64, widths, vec_dtype="f64")
    b64.bind(xs64, ys64)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        b32.spmv()
        b64.spmv()
    t32 = _events_time(b32.spmv, 50, stream)
    t64 = _events_time(b64.spmv, 50, stream)

    def separate():
        for s, x, y in zip(S64, xs64, ys64):
            sellcs.spmv(s, x, y)
    separate()
    tsep = _events_time(separate, 10, stream)
    nnz = sum(A.nnz for A in mats)
    rows = sum(A.nrows for A in mats)
    nbw = sum(A.nrows * w for A, w in zip(mats, widths))
    bytes32 = nnz * 8 + 2 * nbw * 4
    bytes64 = nnz * 12 + 2 * nbw * 8
    cg = sellcs.CG(S64, widths, cpl32=cpl32)
    bs = [torch.from_numpy(B).cuda() for B in Bs]
    xs = [torch.zeros_like(b) for b in bs]
    cg.solve(bs, xs)  # warm-up (graph capture)
    torch.cuda.synchronize()
    t0 = _t.time()
    st32, rel32 = cg.solve(bs, xs)
    torch.cuda.synchronize()
    tts32 = _t.time() - t0
    cg.solve(bs, xs, inner_f64=True, inner_tol=1e-10, max_outer=3)
    torch.cuda.synchronize()
    t0 = _t.time()
    st64, rel64 = cg.solve(bs, xs, inner_f64=True, inner_tol=1e-10, max_outer=3)
    torch.cuda.synchronize()
    tts64 = _t.time() - t0
    return {"systems": len(mats), "rows": rows, "nnz": nnz, "rhs_columns": int(sum(widths)),
            "autotune_s": round(tune_s, 2),
            "tuned_configs": {f"C{C}_sigma{sg}_cpl{cp}": sum(1 for c in cfg if (c["C"], c["sigma"], c["cpl"]) == (C, sg, cp))
                              for C, sg, cp in sorted({(c["C"], c["sigma"], c["cpl"]) for c in cfg})},
            "spmv_batched_f32_us": round(t32 * 1e3, 1), "spmv_batched_f32_GBs": round(bytes32 / t32 / 1e6, 1),
            "spmv_batched_f64_us": round(t64 * 1e3, 1), "spmv_batched_f64_GBs": round(bytes64 / t64 / 1e6, 1),
            "spmv_64_separate_f64_us": round(tsep * 1e3, 1),
            "speedup_batched_f32_vs_separate_f64": round(tsep / t32, 2),
            "speedup_batched_f64_vs_separate_f64": round(tsep / t64, 2),
            "mpcg_time_s": round(tts32, 4), "mpcg_stats": st32, "mpcg_max_rel_residual": float(rel32.max()),
            "f64cg_time_s": round(tts64, 4), "f64cg_stats": st64, "f64cg_max_rel_residual": float(rel64.max()),
            "speedup_mpcg_vs_f64cg": round(tts64 / tts32, 3)}


# ------------------------------------------------------------------ CPU baseline (the oracle)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_call(A, X, Y0, Z0, nthreads=1):
    """One oracle product on the bench workload: the single-thread oracle, or
    its row-parallel OpenMP form on ``nthreads`` host cores."""
    import oracle
    W = WORKLOAD
    kw = dict(alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], y0=Y0, dot_xy=True, dot_yy=True,
              delta=W["delta"], eta=W["eta"], z0=Z0)
    if nthreads > 1:
        r = oracle.spmmv_omp(A, X, nthreads=nthreads, **kw)
        if r is not None:
            return r
    return oracle.spmmv(A, X, **kw)


def _oracle_times(data, nthreads, reps, budget_s):
    """Median seconds of up to ``reps`` oracle calls (at least 3, within budget_s)."""
    A, X, Y0, Z0 = data
    oracle_call(A, X, Y0, Z0, nthreads)
    ts = []
    t_start = time.time()
    while len(ts) < reps and (len(ts) < 3 or time.time() - t_start < budget_s):
        t0 = time.perf_counter()
        oracle_call(A, X, Y0, Z0, nthreads)
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts)), len(ts)


def workload_config(A, nbytes, world):
    return dict(WORKLOAD, nnz=A.nnz, bytes_per_call=nbytes, l2="inputs 0.96 GB > 129 MB L2, no flush",
                parallelism=f"replicas{world}")


def cpu_baseline(data, budget_s=12.0):
    """The oracle on the host: the row-parallel form over all cores (the
    baseline value) and the single-thread form beside it, each the median of
    10 full calls on the bench workload."""
    import oracle
    A = data[0]
    oracle.build()
    nch = (A.nrows + 31) // 32
    nbytes = algorithmic_bytes(A.nnz, A.nrows, A.ncols, nch, nch * 32, 1, 8, 8, True, True, True)
    cores = host_cores()
    omp = oracle.build_omp() is not None and cores > 1
    t1, n1 = _oracle_times(data, 1, 10, budget_s)
    single = {"value": round(nbytes / t1 / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
              "sample": f"median of {n1} full calls of the float64 CSR oracle (Neumaier sums, single thread), "
                        f"{t1:.3f} s each"}
    if not omp:
        return single
    tn, nn = _oracle_times(data, cores, 10, budget_s)
    return {"value": round(nbytes / tn / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"median of {nn} full calls of the float64 CSR oracle with its rows shared among {cores} "
                      f"OpenMP threads (nproc = {cores}), {tn:.4f} s each",
            "single_thread": single}


REF_BUDGET_S = 150.0  # upper bound of the reference arm's warm-up + timed oracle work


def run_reference(args, rank, world):
    """The reference arm: the oracle, as it stands (row-parallel over all host
    cores when OpenMP is available), one full call per step, or a bounded
    row sample per step when the full calls would not end within
    REF_BUDGET_S."""
    import oracle
    oracle.build()
    cores = host_cores()
    nt = cores if oracle.build_omp() is not None else 1
    A, X, Y0, Z0 = make_workload()
    nch = (A.nrows + 31) // 32
    nbytes = algorithmic_bytes(A.nnz, A.nrows, A.ncols, nch, nch * 32, 1, 8, 8, True, True, True)
    # each step one full call, or, when steps x the time of one call would pass
    # REF_BUDGET_S, a bounded sample: the first r rows (the bytes of the call
    # scaled by the sample's share of the nonzeros)
    t1 = time.time()
    oracle_call(A, X, Y0, Z0, nt)
    t_call = time.time() - t1
    sample = "one full oracle call per step"
    if t_call * (args.steps + args.warmup) > REF_BUDGET_S:
        from workloads.generators import CSR
        r = max(4096, int(A.nrows * REF_BUDGET_S / (t_call * (args.steps + args.warmup))))
        e = int(A.rowptr[r])
        nbytes = nbytes * e / A.nnz
        A, Y0, Z0 = CSR(r, A.ncols, A.rowptr[:r + 1], A.col[:e], A.val[:e]), Y0[:r], Z0[:r]
        sample = (f"per step the first {r} rows of the workload ({e} nonzeros; bytes of the full call scaled "
                  f"by the sample's share of the nonzeros)")
    for _ in range(args.warmup):
        oracle_call(A, X, Y0, Z0, nt)
    t0 = time.time()
    for _ in range(args.steps):
        oracle_call(A, X, Y0, Z0, nt)
    dt = (time.time() - t0) / args.steps
    v = round(nbytes / dt / 1e9, 3)
    how = f"rows shared among {nt} OpenMP threads" if nt > 1 else "single thread"
    return {
        "impl": "reference",
        "metric": METRIC,
        "value": v, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": DATA, "config": workload_config(A, nbytes, world),
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": nt, "kind": "oracle",
                         "sample": f"{sample} (float64 CSR oracle, Neumaier sums, {how}; nproc = {cores})"},
        "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------------------------ main


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--powerlaw-config", default=None,
                    help="with --only powerlaw_adjoint: C:sigma:order instead of the autotuner's choice")
    ap.add_argument("--no-fp64-probe", action="store_true",
                    help="skip the float64 rate probe that runs after the timed region")
    ap.add_argument("--only", choices=["laplace", "laplace256", "anderson_w16", "powerlaw_adjoint", "cg_batch", "kpm",
                                       "permuted", "tsm", "fp64_rate", "dist", "layout", "vty"],
                    help="run one secondary workload alone and print its JSON")
    ap.add_argument("--pairs", default=None,
                    help="with --only anderson_w16: comma-separated value:vector precision pairs, e.g. f32:f32; "
                         "with --only tsm: the precisions, e.g. f32")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return

    import torch
    if args.only:
        from paper_1507_08101_gb300 import build
        build.build()
        fns = {"laplace": secondary_laplace, "laplace256": lambda p: secondary_laplace(p, (256,)),
               "fp64_rate": lambda p: measured_fp64_rate(),
               "anderson_w16": lambda p: secondary_anderson(
                   p, [tuple(q.split(":")) for q in args.pairs.split(",")] if args.pairs else None),
               "tsm": lambda p: secondary_tsm(p, tuple(args.pairs.split(",")) if args.pairs else ("f64", "f32")),
               "powerlaw_adjoint": lambda p: secondary_powerlaw(
                   p, args.powerlaw_config.split(":") if args.powerlaw_config else None),
               "cg_batch": secondary_cg_batch, "kpm": secondary_kpm,
               "permuted": secondary_permuted, "dist": secondary_dist,
               "layout": secondary_layout, "vty": secondary_vty}
        print(json.dumps({args.only: fns[args.only](load_peaks()[0])}), flush=True)
        return
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        torch.distributed.init_process_group("nccl")
    from paper_1507_08101_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    result, data = run_ours(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(data)
    if rank == 0 and world == 1 and not args.no_secondary:
        del data
        peak = result["roofline"]["peak"]
        sec = {}
        for name, fn in (("laplace", secondary_laplace), ("anderson_w16", secondary_anderson),
                         ("powerlaw_adjoint", secondary_powerlaw), ("cg_batch", secondary_cg_batch),
                         ("kpm", secondary_kpm), ("vty", secondary_vty),
                         ("tsm", lambda p: secondary_tsm(p, ("f64", "f32"))), ("layout", secondary_layout),
                         ("permuted", secondary_permuted), ("dist", secondary_dist)):
            try:
                sec[name] = fn(peak)
            except Exception as e:  # a failed secondary measurement must not hide the headline
                sec[name] = {"error": f"{type(e).__name__}: {e}"}
        result["secondary"] = sec
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
