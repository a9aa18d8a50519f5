"""Host-side helpers of the benchmark (no GPU): the traffic record is used only
while the kernel code it was measured on is unchanged -- comments aside -- and
for the same matrix size."""
import json
import os
import shutil
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2310_13421_gb300 import synth  # noqa: E402


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
    with open(os.path.join(ROOT, "profiles", "traffic_k_pass_fixed_n13.json")) as fh:
        rec = json.load(fh)
    current = rec["kernel_digest"] == bench.kernel_digest()
    mean = float(np.mean(rec["bytes_per_launch_captured"]))
    assert bench.measured_traffic(14) == (4 * mean if current else None)
    assert bench.measured_traffic(13) == (mean if current else None)
    assert bench.measured_traffic(12) is None              # no scaling down from the captured size
    # DRAM traffic of a pass launch near its algorithmic bytes (no re-reads):
    # within 2 % on average, 5 % per launch (writes still in L2 when a launch
    # ends are counted by the next one)
    alg = rec["algorithmic_bytes_per_launch_captured"]
    assert abs(mean / alg - 1) < 0.02
    for b in rec["bytes_per_launch_captured"]:
        assert abs(b / alg - 1) < 0.05


def test_accuracy_rows_follow_the_rc_layout():
    # the oracle's weights laid out in RC order (weight of string t at row
    # bits = z, column bits = x xor z), read back by the bench's sampler, are
    # the oracle's own X-rows; the accuracy leg then reports zero error, and a
    # complex64 input gives the same rows through the gathered-diagonal path
    import oracle
    from _helpers import rc_positions
    n = 6
    A = synth.hermitian(n, seed=11)
    W = np.empty(4 ** n, dtype=np.complex128)
    W[rc_positions(n)] = oracle.coeffs_fwht(A)
    xs = bench.accuracy_xs(n, count=8)
    got = bench.rows_of(W.reshape(2 ** n, 2 ** n), n, xs)
    assert np.array_equal(got, oracle.coeffs_xrows(A, xs))
    acc = bench.oracle_accuracy(A, n, xs, {"exact": got})["exact"]
    assert acc["normwise"] == 0 and acc["max_over_m_x"] == 0
    A32 = A.astype(np.complex64)
    assert np.array_equal(oracle.coeffs_xrows(A32, xs), oracle.coeffs_xrows(A32.astype(np.complex128), xs))


def test_weyl_rows_follow_the_kernel_layout():
    # the Weyl oracle's weights placed where the kernel puts them (row digits
    # b, column digits a + b mod d), read back at the bench's positions, are
    # the oracle's rows of the sampled shifts: zero error in the accuracy leg
    from oracle import core
    d, n = 3, 4
    N = d ** n
    A = synth.hermitian_side(N, seed=5)
    c = core.weyl_coeffs_dft(A, d)
    W = np.empty((N, N), dtype=np.complex128)
    a = np.repeat(np.arange(N), N)
    b = np.tile(np.arange(N), N)
    W[b, bench._digit_add(a, b, d, n)] = c.reshape(-1)
    a_s = np.array([0, 5, N - 1])
    bb = np.arange(N)
    got = np.stack([W[bb, bench._digit_add(bb, np.full(N, x), d, n)] for x in a_s])
    assert np.array_equal(got, c[a_s])
    acc = bench.weyl_accuracy(A, d, a_s, {"exact": got})["exact"]
    assert acc["normwise"] == 0.0


def test_gellmann_accuracy_leg_reads_labels_at_their_positions():
    # the Gell-Mann oracle's coefficients sit at row r, column c of their
    # label (the kernel's layout): read back at the bench's sampled labels
    # they give zero error, and a perturbed one a positive weighted error
    from oracle import core
    d, n = 3, 4
    N = d ** n
    A = synth.hermitian_side(N, seed=6)
    g = core.gellmann_coeffs(A, d)
    rows, cols = np.array([0, N - 1, 0, 7, 40]), np.array([0, N - 1, N - 1, 3, 40])
    acc = bench.gellmann_accuracy(A, d, rows, cols, {"exact": g[rows, cols]})["exact"]
    assert acc["normwise_weighted"] == 0.0 and acc["coefficients"] == 5
    bad = g[rows, cols].copy()
    bad[1] += 1e-6
    assert bench.gellmann_accuracy(A, d, rows, cols, {"bad": bad})["bad"]["normwise_weighted"] > 0
