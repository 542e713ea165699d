"""The committed ncu evidence matches the committed kernels: every DRAM-traffic
entry that bench.py reports resolves against the current kernel sources (its
source hash), names a summary that exists, and every ncu command written in
the summaries leaves the GPU clocks alone (--clock-control none)."""
import glob
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# the kinds that can lead the headline's profile, and the launches the bench
# line reports beside it (persistent batch, emulated FP64 GEMM)
REPORTED = ("chol", "gemm_simt_f32", "tc_gemm", "oz_gemm", "batch")


def test_traffic_entries_match_the_current_kernel_sources():
    for kind in REPORTED:
        tr = bench._traffic_for(kind, bench.KIND_SOURCES[kind])
        assert tr is not None, f"{kind}: no ncu traffic for the current source (re-capture it)"
        assert tr[0] > 0
        m = re.search(r"profiles/[\w.]+\.md", tr[1])
        assert m and os.path.exists(os.path.join(ROOT, m.group(0))), tr[1]


def test_every_ncu_command_keeps_the_clocks():
    files = glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt"))
    assert files
    for path in files:
        text = open(path).read().replace("\\\n", " ")   # join continued command lines
        for line in text.splitlines():
            if re.match(r"\s*(\S+\s*&&\s*)?ncu\s+-", line) or re.search(r"&&\s*ncu\s+-", line):
                assert "--clock-control none" in line, f"{os.path.basename(path)}: {line.strip()[:120]}"


def test_roofline_arithmetic():
    """achieved = the launches' method flops (bytes for streaming kinds) over
    their summed device time; each kind against its own peak."""
    peaks = (1940.0e3, 1728.0e3, 6800.0, "measured")   # BF16 burst / sustained GFLOP/s, HBM GB/s
    rec = {"ms": 2.0, "flops": 4.0e9, "bytes": 1.0e9, "launches": 4}
    expect = {"chol": bench.FP64_SM_PEAK_GFLOPS, "gemm_simt": bench.FP64_PEAK_GFLOPS,
              "gemm_simt_f32": bench.FP32_PEAK_GFLOPS, "tc_gemm": 1728.0e3,
              "oz_gemm": 1728.0e3 / bench.OZ_PAIRS}
    for kind, peak in expect.items():
        r = bench.roofline_of(kind, rec, peaks)
        assert r["achieved"] == 4.0e9 / 2.0e-3 / 1e9 and r["unit"] == "GFLOP/s"
        assert r["peak"] == peak and abs(r["frac"] - r["achieved"] / peak) < 1e-12
        assert r["flops_per_launch"] == 1.0e9 and r["bytes_per_launch"] == 2.5e8
    r = bench.roofline_of("stream", rec, peaks)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["achieved"] == 1.0e9 / 2.0e-3 / 1e9
    assert abs(r["frac"] - r["achieved"] / 6800.0) < 1e-12
