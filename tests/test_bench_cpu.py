"""Host logic of bench.py that needs no GPU: the algorithmic byte count of a
call (padding excluded, each term where the contract puts it), the float64
flop count, and the rule that a recorded ncu traffic figure is reported only
while the kernel source it was taken on is unchanged."""
import os
import shutil

import bench


def test_algorithmic_bytes_terms():
    nnz, n, m, nch, nsl = 1000, 100, 120, 4, 128
    base = bench.algorithmic_bytes(nnz, n, m, nch, nsl, 1, 8, 8, False, False, False)
    # values + int32 indices once, x once, y written once, chunk offsets and slot lengths
    assert base == nnz * 12 + m * 8 + n * 8 + nch * 8 + nsl * 4
    # the beta term reads y once more; the chain reads and writes z; the permutation is one int per slot
    assert bench.algorithmic_bytes(nnz, n, m, nch, nsl, 1, 8, 8, True, False, False) - base == n * 8
    assert bench.algorithmic_bytes(nnz, n, m, nch, nsl, 1, 8, 8, False, True, False) - base == 2 * n * 8
    assert bench.algorithmic_bytes(nnz, n, m, nch, nsl, 1, 8, 8, False, False, True) - base == nsl * 4
    # vectors scale with the block width, the matrix stream does not
    w4 = bench.algorithmic_bytes(nnz, n, m, nch, nsl, 4, 8, 8, False, False, False)
    assert w4 - base == 3 * (m + n) * 8
    # float32 values and vectors
    f32 = bench.algorithmic_bytes(nnz, n, m, nch, nsl, 1, 4, 4, False, False, False)
    assert base - f32 == nnz * 4 + (m + n) * 4


def test_fp64_flops():
    # row sums: 2 per nonzero and column; epilogue per row and column:
    # shift 2, scale 1, beta 2, each dot 2, chain 3
    assert bench.fp64_flops(10, 3, 1, False, False, False, 0, False) == 20
    assert bench.fp64_flops(10, 3, 2, True, True, True, 2, True) == 2 * 10 * 2 + (2 + 1 + 2 + 4 + 3) * 3 * 2


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1507_08101_gb300", "csrc")
    csrc = tmp_path / "paper_1507_08101_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for fn in ("spmv_kernel.cuh", "spmv_launch.cuh"):
        shutil.copy(os.path.join(src, fn), csrc / fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.kernel_source_hash()
    (tmp_path / "profiles" / "k.md").write_text(f"traffic_bytes_per_launch: 12345 kernel_src_sha: {sha}\n")
    assert bench.recorded_traffic("k.md") == 12345.0
    assert bench.recorded_traffic("missing.md") is None
    # any change to the kernel source voids the recorded figure
    with open(csrc / "spmv_kernel.cuh", "a") as f:
        f.write("\n")
    assert bench.recorded_traffic("k.md") is None


def test_whole_job_rate():
    # every rank (a replica) processes the units in the slowest rank's time
    assert bench.whole_job_rate(1e9, 2.0, 4) == 4e9 / 2e-3
