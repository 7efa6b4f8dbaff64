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
        ms = ev0.elapsed_time(ev1)
        ms_step = ms / args.steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
            ms_step = ms / args.steps

        # e2e: host (pinned) buffers, H2D of x, y, z and D2H of y, z, dots inside the timed region
        hx_h = torch.from_numpy(X).pin_memory()
        hy_h = torch.from_numpy(Y0).pin_memory()
        hz_h = torch.from_numpy(Z0).pin_memory()
        oy = torch.empty_like(hy_h).pin_memory()
        oz = torch.empty_like(hz_h).pin_memory()
        od = torch.empty(3, dtype=torch.float64).pin_memory()

        def e2e_step():
            x.copy_(hx_h, non_blocking=True)
            y.copy_(hy_h, non_blocking=True)
            z.copy_(hz_h, non_blocking=True)
            step()
            oy.copy_(y, non_blocking=True)
            oz.copy_(z, non_blocking=True)
            od.copy_(dot, non_blocking=True)

        for _ in range(max(1, args.warmup)):
            e2e_step()
        stream.synchronize()
        e2e_steps = max(3, min(args.steps, 20))
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev2.record(stream)
        for _ in range(e2e_steps):
            e2e_step()
        ev3.record(stream)
        torch.cuda.synchronize()
        e2e_ms = ev2.elapsed_time(ev3) / e2e_steps
        h2d = X.nbytes + Y0.nbytes + Z0.nbytes
        d2h = Y0.nbytes + Z0.nbytes + 3 * 8
        for h in (hx, hy, hz):
            sellcs.sp_dense_destroy(h)

    gbs = nbytes / (ms_step * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    result = {
        "metric": "SpMMV effective HBM GB/s (augmented SELL-32-256, f64, irregular N=2^21)",
        "value": round(gbs * world, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded irregular band matrix standing in for the paper's SuiteSparse inputs)",
        "config": dict(W, nnz=A.nnz, nstored=info["nstored"], bytes_per_call=nbytes,
                       l2="inputs 0.96 GB > 129 MB L2, no flush", parallelism=f"replicas{world}"),
        "roofline": {"bound": "hbm", "achieved": round(gbs, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                     "traffic": recorded_traffic("k_spmmv_irregular_augmented.md"),
                     "kernel": "k_spmmv<double,double,1,true>", "algorithmic_bytes_per_launch": nbytes},
        "e2e": {"value": round(nbytes / (e2e_ms * 1e-3) / 1e9 * world, 2), "unit": "GB/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 4)},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
        "setup": {"sell_build_s": round(setup_s, 4), "in_spmv_calls": round(setup_s / (ms_step * 1e-3), 1)},
    }
    return result, (A, X, Y0, Z0)


# ------------------------------------------------------------------ CPU baseline (the oracle)


def oracle_call(A, X, Y0, Z0):
    import oracle
    W = WORKLOAD
    return oracle.spmmv(A, X, alpha=W["alpha"], gamma=W["gamma"], beta=W["beta"], y0=Y0, dot_xy=True, dot_yy=True,
                        delta=W["delta"], eta=W["eta"], z0=Z0)


def cpu_baseline(data, budget_s=12.0):
    import oracle
    A, X, Y0, Z0 = data
    oracle.build()
    nch = (A.nrows + 31) // 32
    nbytes = algorithmic_bytes(A.nnz, A.nrows, A.ncols, nch, nch * 32, 1, 8, 8, True, True, True)
    oracle_call(A, X, Y0, Z0)
    t0 = time.time()
    n = 0
    while time.time() - t0 < budget_s and n < 50:
        oracle_call(A, X, Y0, Z0)
        n += 1
    dt = (time.time() - t0) / n
    return {"value": round(nbytes / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} full calls of the float64 CSR oracle (Neumaier sums, single thread) on the same "
                      f"workload, {dt:.3f} s each"}


def run_reference(args, rank, world):
    """The reference arm: the oracle, as it stands, on the host cores."""
    import oracle
    oracle.build()
    A, X, Y0, Z0 = make_workload()
    nch = (A.nrows + 31) // 32
    nbytes = algorithmic_bytes(A.nnz, A.nrows, A.ncols, nch, nch * 32, 1, 8, 8, True, True, True)
    for _ in range(args.warmup):
        oracle_call(A, X, Y0, Z0)
    t0 = time.time()
    for _ in range(args.steps):
        oracle_call(A, X, Y0, Z0)
    dt = (time.time() - t0) / args.steps
    v = round(nbytes / dt / 1e9, 3)
    return {
        "impl": "reference",
        "metric": "SpMMV effective HBM GB/s (augmented SELL-32-256, f64, irregular N=2^21)",
        "value": v, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": dict(WORKLOAD, nnz=A.nnz, bytes_per_call=nbytes),
        "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": "one full oracle call per step (float64 CSR, Neumaier sums, single thread)"},
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
    ap.add_argument("--extra", action="store_true", help="also run the secondary workloads")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return

    import torch
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
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
