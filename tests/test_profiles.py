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
