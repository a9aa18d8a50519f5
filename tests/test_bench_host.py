"""Host-side helpers of the benchmark (no GPU): the traffic record is used only
while the kernel code it was measured on is unchanged -- comments aside -- and
for the same matrix size."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_only_drops_comments_and_blank_space():
    a = "int f(int x) {  // doubles x\n  return 2 * x; /* the\n result */\n}\n"
    b = "int f(int x)\n{\n  return 2 * x;\n}"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(a.replace("2 * x", "3 * x"))


def test_kernel_digest_ignores_comments_but_not_code(tmp_path):
    src = os.path.join(ROOT, "paper_2310_13421_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    d0 = bench.kernel_digest(str(dst))
    assert d0 == bench.kernel_digest()
    p = dst / "tpd_pass.cuh"
    text = p.read_text()
    p.write_text(text + "\n// a comment only\n")
    assert bench.kernel_digest(str(dst)) == d0
    p.write_text(text.replace("constexpr uint32_t kFull", "constexpr uint32_t kFull2", 1))
    assert bench.kernel_digest(str(dst)) != d0


def test_traffic_record_used_only_for_its_kernels_and_size():
    with open(os.path.join(ROOT, "profiles", "traffic_n14_c128.json")) as fh:
        rec = json.load(fh)
    current = rec["kernel_digest"] == bench.kernel_digest()
    assert bench.measured_traffic(14) == (rec["bytes_per_launch"] if current else None)
    assert bench.measured_traffic(13) is None
    # DRAM traffic of a pass launch within 1 % of its algorithmic bytes (no re-reads)
    assert abs(rec["bytes_per_launch"] / rec["algorithmic_bytes_per_launch"] - 1) < 0.01
