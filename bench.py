#!/usr/bin/env python
"""Benchmark of the GB300 tensorized Pauli decomposition (arXiv:2310.13421).

Workload (the metric's configuration): one dense 16384 x 16384 complex128
random Hermitian matrix (n = 14 qubits, 4.29 GB, above L2), decomposed in
place into its 4^14 Pauli weights.  One step = one full decomposition (all
passes) of the resident matrix; the pristine input is restored between steps
outside the timed events.

Prints ONE JSON line (rank 0).  `value` = Pauli coeffs/s over all ranks with
inputs resident in HBM; `e2e` = the same metric through the C ABI with host
buffers (pinned), every step's host<->device copies inside the timed region
(steps alternate over three streams with their own buffers, so one step's
copies overlap another's); `roofline` = achieved HBM bandwidth of the pass
kernel (algorithmic bytes: read + write of the matrix per pass launch)
against the measured copy peak; `paper_arithmetic` = the same metric with
IEEE fp64 adds rounded per level; `cpu_baseline` = the CPU oracle timed on a
bounded sample; `extra` = the complex64 plain / compensated / fixed-point
forms at n = 15 beside the complex128 ones, the errors of every form against
the fp64 oracle, the batch of 4096 matrices, the partial decomposition, zero
skipping, sparse input, composition, autograd, the layout and norm helpers,
the Weyl and generalized Gell-Mann bases (d = 3, n = 9) and the paper's
Alg. 2 on the host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Pauli coeffs/s & HBM GB/s (n=14 c128); fp32-compensated vs fp64 speedup"
UNIT = "coeffs/s"
N_QUBITS = 14
SEED = 1002


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-extra", action="store_true", help="skip the fp64 / complex64 comparison runs")
    p.add_argument("--e2e-steps", type=int, default=8)
    p.add_argument("--e2e-streams", type=int, default=3, help="streams the end-to-end steps alternate over")
    p.add_argument("--qubits", type=int, default=N_QUBITS,
                   help="matrix size of the timed workload (14 = the metric's workload; smaller for profiling)")
    p.add_argument("--no-batch", action="store_true", help="skip the batch-of-4096 comparison run")
    p.add_argument("--workload", choices=["dense", "batch", "weyl", "gellmann"], default="dense",
                   help="dense: the metric's n=14 matrix (default); batch: only the batch comparison "
                        "(--batch-count matrices, n ~ U{3..10}); weyl / gellmann: only the Weyl- or "
                        "Gell-Mann-basis row (--weyl-n qutrits); e.g. for profiling")
    p.add_argument("--batch-count", type=int, default=4096)
    p.add_argument("--weyl-n", type=int, default=9, help="qutrits of the --workload weyl matrix")
    p.add_argument("--storage", choices=["c128", "c64"], default="c128",
                   help="dense workload storage (c128 = the metric's; c64 for profiling the fp32 forms)")
    p.add_argument("--precision", choices=["default", "fixed", "plain", "compensated"], default="default")
    return p.parse_args()


def dist_env():
    from paper_2310_13421_gb300.dist import rank_env
    return rank_env()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = [num(r[1]) for r in rows]
        mx = [num(r[2]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s, p in zip(sm, (num(r[3]) for r in rows)) if p > 200] or sm
        return {"sm_mhz": float(np.nanmedian(loaded)), "sm_max_mhz": float(np.nanmax(mx)),
                "reasons": reasons, "samples": len(rows),
                "power_w_max": float(np.nanmax([num(r[3]) for r in rows]))}


# ------------------------------------------------------------------ oracle timing

def oracle_rate(A, n, budget_s=12.0):
    """CPU oracle (Walsh-Hadamard form, all host cores) on a bounded sample of
    X-rows of the same matrix: returns (coeffs/s, cores, sample text)."""
    import oracle
    N = 2 ** n
    rng = np.random.default_rng(0)
    order = rng.permutation(N).astype(np.uint64)
    done, t0, chunk = 0, time.perf_counter(), 256
    while done < N and time.perf_counter() - t0 < budget_s:
        xs = order[done:done + chunk]
        oracle.coeffs_xrows(A, xs)
        done += len(xs)
        chunk = min(chunk * 2, 4096)
    dt = time.perf_counter() - t0
    return done * N / dt, oracle.num_threads(), "%d of %d X-rows (all %d Z-masks each) of the n=%d matrix, %.1f s" % (
        done, N, N, n, dt)


# ------------------------------------------------------------------ reference arm

def run_reference(args, world, rank):
    if rank != 0:
        return 0
    from paper_2310_13421_gb300 import synth
    import oracle
    n = N_QUBITS
    A = synth.hermitian(n, seed=SEED)
    N = 2 ** n
    rows_per_step = 512
    rng = np.random.default_rng(1)
    for _ in range(args.warmup):
        oracle.coeffs_xrows(A, rng.integers(0, N, size=64).astype(np.uint64))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.coeffs_xrows(A, rng.integers(0, N, size=rows_per_step).astype(np.uint64))
    dt = time.perf_counter() - t0
    value = args.steps * rows_per_step * N / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "n=14 dense Hermitian complex128, 16384x16384 (CPU oracle, Walsh-Hadamard form)",
                   "sample_per_step": "%d X-rows x %d Z-masks" % (rows_per_step, N)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": "%d steps of %d random X-rows each" % (args.steps, rows_per_step)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ our arm

KERNEL_SOURCES = ("tpd_pass.cuh", "tpd_arith.cuh", "tpd_plan.h", "tpd_shape.h", "tpd_launch.h", "tpd_planner.cpp",
                  "tpd_kernels_impl.cuh", "tpd_kernels_fixed_dec.cu", "tpd_kernels_fixed_com.cu",
                  "tpd_kernels_shapes_fixed.cu", "tpd_kernels_c128.cu")


def _code_only(text):
    """C/C++ source without comments and blank space (a comment edit leaves
    the compiled kernels, and so the recorded traffic, unchanged)."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_digest(csrc=None):
    """Hash of the code (comments excluded) that decides the complex128 pass
    kernels and their plans."""
    h = hashlib.sha256()
    csrc = csrc or os.path.join(ROOT, "paper_2310_13421_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f in KERNEL_SOURCES:
            with open(os.path.join(csrc, f), encoding="utf-8") as fh:
                h.update(f.encode() + _code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def measured_traffic(n):
    """Per-launch DRAM bytes of the complex128 fixed-point pass kernel at n
    qubits, from the committed small-case ncu record (n = 13) scaled by the
    elements a launch reads and writes (4^(n - 13)), if that record was taken
    on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "traffic_k_pass_fixed_n13.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    m = d.get("captured_qubits")
    if d.get("kernel_digest") != kernel_digest() or not isinstance(m, int) or n < m:
        return None
    per = d.get("bytes_per_launch_captured") or []
    if not per:
        return None
    return float(np.mean(per)) * 4.0 ** (n - m)


def time_decompose(tpd, L, torch, work, pristine, n, steps, warmup, precision, stream):
    """Per-step and per-pass device times (ms) of in-place decompositions."""
    code = L.TPD_C128 if work.dtype == torch.complex128 else L.TPD_C64
    npass = L.tpd_plan_describe(n, code, L.options(precision=precision))[0]
    nev = max(npass, 1) + 1
    wsb = L.tpd_workspace_size(n, code, L.options(precision=precision))
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device=work.device)
    for _ in range(warmup):
        work.copy_(pristine)
        st = L.tpd_decompose(work.data_ptr(), n, code, L.options(precision=precision), ws.data_ptr(), wsb,
                             stream.cuda_stream)
        assert st == 0, L.status_string(st)
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nev)] for _ in range(steps)]
    for row in evs:            # torch creates the CUDA event on first record
        for e in row:
            e.record(stream)
    torch.cuda.synchronize()
    for k in range(steps):
        work.copy_(pristine)                       # restore, outside the events
        opt = L.options(precision=precision, pass_events=[e.cuda_event for e in evs[k]])
        st = L.tpd_decompose(work.data_ptr(), n, code, opt, ws.data_ptr(), wsb, stream.cuda_stream)
        assert st == 0, L.status_string(st)
    torch.cuda.synchronize()
    step_ms = [evs[k][0].elapsed_time(evs[k][-1]) for k in range(steps)]
    pass_ms = [[evs[k][p].elapsed_time(evs[k][p + 1]) for p in range(nev - 1)] for k in range(steps)]
    return step_ms, pass_ms, npass


def time_batch(tpd, L, torch, stream, count=4096, seed=1004, reps=5):
    """Batch of `count` random Hermitian complex128 matrices, n_i ~ U{3..10}:
    the batched call in its two forms, each captured in a CUDA graph -- one
    launch per (qubit count, pass) (default) and one persistent kernel launch
    for the whole batch (variant 2) -- against one tpd_decompose call per matrix on the
    same stream.  All matrices live in one buffer, restored from a pristine
    copy between repetitions outside the timed events."""
    from paper_2310_13421_gb300 import synth
    ns = [int(x) for x in synth.batch_sizes(count, seed=seed)]
    offs = np.concatenate([[0], np.cumsum([4 ** n for n in ns])]).astype(np.int64)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    buf = torch.randn(int(offs[-1]), dtype=torch.complex128, device="cuda", generator=g) * np.sqrt(2.0)
    mats = [buf[offs[i]:offs[i + 1]].view(2 ** n, 2 ** n) for i, n in enumerate(ns)]
    for m in mats:                           # A = (B + B^H) / 2
        m.copy_((m + m.mH) * 0.5)
    pristine = buf.clone()
    passes = {n: max(L.tpd_plan_describe(n, L.TPD_C128, L.options())[0], 1) for n in set(ns)}
    alg_bytes = sum(32 * passes[n] * 4 ** n for n in ns)
    graphs = {}
    batches = {}
    for name, variant in (("persistent", 2), ("per_pass", 0)):
        batch = tpd.Batch(mats, variant=variant)
        batch.decompose()                    # plans and kernel attributes, outside the capture
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            batch.decompose()
        graphs[name], batches[name] = graph, batch
    wsb = max(L.tpd_workspace_size(n, L.TPD_C128, L.options()) for n in set(ns))
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")

    def loop():
        for m, n in zip(mats, ns):
            st = L.tpd_decompose(m.data_ptr(), n, L.TPD_C128, None, ws.data_ptr(), wsb, stream.cuda_stream)
            assert st == 0, L.status_string(st)

    # the autotuner's choice for this very batch (never slower than the
    # planner's defaults on it), captured the same way
    from paper_2310_13421_gb300 import autotune
    tuned = autotune.tune_batch(mats)
    buf.copy_(pristine)
    batch = tpd.Batch(mats, variant=tuned["variant"])
    batch.decompose()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.decompose()
    graphs["autotuned"], batches["autotuned"] = graph, batch

    res = {}
    for name, fn in (("persistent", graphs["persistent"].replay), ("per_pass", graphs["per_pass"].replay),
                     ("autotuned", graphs["autotuned"].replay), ("per_matrix_loop", loop)):
        times = []
        for k in range(reps + 2):
            buf.copy_(pristine)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            if k >= 2:
                times.append(e0.elapsed_time(e1))
        res[name] = float(np.median(times))
    # the three forms agree exactly (same exact sums, one rounding per output)
    outs = []
    for fn in (graphs["persistent"].replay, graphs["per_pass"].replay, graphs["autotuned"].replay, loop):
        buf.copy_(pristine)
        fn()
        outs.append(buf.clone())
    same = bool(all(torch.equal(outs[0], o) for o in outs[1:]))
    status = batches["persistent"].status()
    L.tpd_tune_clear()
    del buf, pristine, outs, mats, batches, graphs
    torch.cuda.empty_cache()
    ms = res["autotuned"]                    # the autotuner's choice for this batch
    return {"matrices": count, "n_range": [3, 10], "data_bytes": int(offs[-1]) * 16,
            "algorithmic_bytes": alg_bytes, "graph_ms": ms, "matrices_per_s": count / (ms * 1e-3),
            "coeffs_per_s": int(offs[-1]) / (ms * 1e-3), "hbm_gbs": alg_bytes / (ms * 1e-3) / 1e9,
            "per_pass_graph_ms": res["per_pass"],
            "one_launch_graph_ms": res["persistent"],
            "one_launch_hbm_gbs": alg_bytes / (res["persistent"] * 1e-3) / 1e9,
            "autotuned_graph_ms": res["autotuned"],
            "autotuned_choice": {"per_n": {str(k): v for k, v in tuned["per_n"].items()},
                                 "batch_form": "one persistent launch" if tuned["variant"] == 2
                                 else "one launch per (qubit count, pass)"},
            "per_matrix_loop_ms": res["per_matrix_loop"],
            "speedup_vs_loop": res["per_matrix_loop"] / ms, "identical_results": same, "one_launch_status": status}


def _event_ms(torch, stream, fn, reps=5, setup=None):
    times = []
    for k in range(reps + 2):
        if setup is not None:
            setup()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def _digit_add(x, y, d, n):
    """digit-wise (x + y) mod d of base-d integers (arrays)"""
    out, p = np.zeros_like(x), 1
    for _ in range(n):
        out += ((x // p) % d + (y // p) % d) % d * p
        p *= d
    return out


def time_weyl(tpd, L, torch, stream, d=3, n=9, seed=1006, shifts=8):
    """Decomposition in the Weyl (clock-and-shift) basis of n qudits of
    dimension d (the basis Sec. V names): a random d^n x d^n Hermitian matrix,
    complex128 (block fixed point, and fp64) and complex64 (fp32), one launch per qudit
    level, each reading and writing the whole matrix.  Returns the timings
    and, for the accuracy leg, the weights of a few shifts a (row digits b,
    column digits a + b) of each result."""
    from paper_2310_13421_gb300 import synth
    N = d ** n
    A = synth.hermitian_side(N, seed)
    rng = np.random.default_rng(seed)
    a_s = np.array([0, 1, N - 1] + [int(v) for v in rng.integers(0, N, shifts - 3)], dtype=np.int64)
    b = np.arange(N, dtype=np.int64)
    pos = np.concatenate([b * N + _digit_add(b, np.full(N, a), d, n) for a in a_s])
    out, rows = {"d": d, "n": n, "side": N}, {}
    legs = (("c128", torch.complex128, L.TPD_C128, 16, L.TPD_PREC_DEFAULT,
             "int64 block fixed point, one binary point per class of d summed elements"),
            ("c128_fp64", torch.complex128, L.TPD_C128, 16, L.TPD_PREC_PLAIN, "fp64, rounded every level"),
            ("c64", torch.complex64, L.TPD_C64, 8, L.TPD_PREC_DEFAULT, "fp32, rounded every level"))
    for name, tt, code, elem, prec, arith in legs:
        src = torch.from_numpy(A).to("cuda", tt)
        work = torch.empty_like(src)
        opt = L.options(precision=prec)

        def step():
            st = L.tpd_weyl_decompose(work.data_ptr(), n, d, code, opt, stream.cuda_stream)
            assert st == 0, L.status_string(st)

        ms = _event_ms(torch, stream, step, setup=lambda: work.copy_(src))
        alg = 2 * n * N * N * elem
        out[name] = {"ms": ms, "coeffs_per_s": N * N / (ms * 1e-3), "hbm_gbs_algorithmic": alg / (ms * 1e-3) / 1e9,
                     "launches": n, "arithmetic": arith}
        rows[name] = work.reshape(-1).index_select(0, torch.from_numpy(pos).cuda()).cpu().numpy() \
            .astype(np.complex128).reshape(len(a_s), N)
        del src, work
        torch.cuda.empty_cache()
    return out, (A, d, a_s, rows)


def weyl_accuracy(A, d, a_s, results):
    """Accuracy leg for the Weyl basis: the sampled shifts' weights against
    the Weyl oracle (fp64) on the same matrix, normwise over the sample."""
    from oracle import core
    want = core.weyl_rows(A, d, a_s)
    return {name: {"normwise": float(np.linalg.norm(got - want) / np.linalg.norm(want)), "weights": int(want.size)}
            for name, got in results.items()}


def time_gellmann(tpd, L, torch, stream, d=3, n=9, seed=1007, labels=256, A=None):
    """Decomposition in the generalized Gell-Mann basis of n qudits of
    dimension d (the other basis Sec. V names): a random d^n x d^n Hermitian
    matrix (or the given one), complex128 (fp64) and complex64 (fp32), one
    launch per qudit level, each reading and writing the whole matrix.
    Returns the timings and, for the accuracy leg, the coefficients of a
    sample of labels (r, c) of each result."""
    from paper_2310_13421_gb300 import synth
    N = d ** n
    if A is None:
        A = synth.hermitian_side(N, seed)
    rng = np.random.default_rng(seed)
    rows_, cols_ = rng.integers(0, N, labels), rng.integers(0, N, labels)
    rows_[:3], cols_[:3] = (0, N - 1, 0), (0, N - 1, N - 1)
    pos = torch.from_numpy(rows_ * N + cols_)
    out, got = {"d": d, "n": n, "side": N}, {}
    legs = (("c128", torch.complex128, L.TPD_C128, 16, "fp64, rounded every level"),
            ("c64", torch.complex64, L.TPD_C64, 8, "fp32, rounded every level"))
    for name, tt, code, elem, arith in legs:
        src = torch.from_numpy(A).to("cuda", tt)
        work = torch.empty_like(src)

        def step():
            st = L.tpd_gellmann_decompose(work.data_ptr(), n, d, code, None, stream.cuda_stream)
            assert st == 0, L.status_string(st)

        ms = _event_ms(torch, stream, step, setup=lambda: work.copy_(src))
        alg = 2 * n * N * N * elem
        imag_max = float(work.imag.abs().max().item())
        out[name] = {"ms": ms, "coeffs_per_s": N * N / (ms * 1e-3), "hbm_gbs_algorithmic": alg / (ms * 1e-3) / 1e9,
                     "launches": n, "arithmetic": arith, "hermitian_input_max_abs_imag": imag_max}
        got[name] = work.reshape(-1).index_select(0, pos.cuda()).cpu().numpy().astype(np.complex128)
        del src, work
        torch.cuda.empty_cache()
    return out, (A, d, rows_, cols_, got)


def gellmann_accuracy(A, d, rows_, cols_, results):
    """Accuracy leg for the Gell-Mann basis: the sampled labels' coefficients
    against the Gell-Mann oracle (fp64) on the same matrix, in the weighted
    norm sqrt(sum tr(G^2) |g|^2) over the sample."""
    from oracle import core
    want = core.gellmann_coeffs_at(A, d, rows_, cols_)
    n = int(round(np.log(A.shape[0]) / np.log(d)))
    w = np.ones(len(rows_))
    r, c = np.array(rows_), np.array(cols_)
    for _ in range(n):
        w *= np.where((r % d == 0) & (c % d == 0), float(d), 2.0)
        r, c = r // d, c // d
    w = np.sqrt(w)
    return {name: {"normwise_weighted": float(np.linalg.norm(w * (got - want)) / np.linalg.norm(w * want)),
                   "coefficients": int(want.size)} for name, got in results.items()}


def alg2_baseline(A, W_rc, n, samples=1 << 20):
    """The paper's algorithm on the host over the whole matrix -- the
    iterative form (Alg. 2, the CMWs of Eq. 4 level by level in place) on one
    host thread and on all host cores: coeffs/s, and the largest deviation
    from the GPU result on a random sample of strings."""
    import oracle
    rng = np.random.default_rng(7)
    s = rng.integers(0, 4 ** n, size=samples, dtype=np.int64)
    r = np.zeros_like(s)
    c = np.zeros_like(s)
    for beta in range(n):
        t = (s >> (2 * beta)) & 3
        r |= (t >> 1) << beta
        c |= (t & 1) << beta
    gpu = W_rc.reshape(-1)[(r << n) | c]
    out = {}
    for key, threads in (("alg2_1thread", 1), ("alg2", 0)):
        t0 = time.perf_counter()
        w = oracle.tpd_alg2(A, threads=threads)
        dt = time.perf_counter() - t0
        dev = float(np.max(np.abs(gpu - w[s])) / np.max(np.abs(w)))
        out[key] = {"value": 4 ** n / dt, "unit": UNIT, "seconds": dt,
                    "threads": threads or oracle.num_threads(),
                    "kind": "the paper's iterative TPD (Alg. 2) on the host, in place, fp64, whole matrix",
                    "max_rel_dev_vs_gpu_sampled": dev}
        del w
    return out


def time_partial(tpd, L, torch, stream, n=14, seed=1005):
    """Partial decomposition (Alg. 3) of the planted n=14 Heisenberg chain
    for its 53 strings, against the full decomposition of the same matrix."""
    from paper_2310_13421_gb300 import synth
    J, h = synth.heisenberg_params(n, seed=seed)
    H = torch.from_numpy(synth.heisenberg(n, J, h)).cuda()
    terms = synth.heisenberg_terms(n, J, h)
    strings = [synth.string_index(t) for t in terms]
    want = torch.tensor([terms[t] for t in terms], dtype=torch.complex128)
    work = torch.empty_like(H)
    part = tpd.Partial(n, strings)
    out = torch.empty(len(strings), dtype=torch.complex128, device="cuda")
    ms_part = _event_ms(torch, stream, lambda: part.decompose(work, inplace=True, out=out),
                        setup=lambda: work.copy_(H))
    exact = bool(torch.equal(out.cpu(), want))
    ms_full = _event_ms(torch, stream, lambda: tpd.decompose(work, inplace=True), setup=lambda: work.copy_(H))
    del H, work
    torch.cuda.empty_cache()
    return {"strings": len(strings), "partial_ms": ms_part, "full_ms": ms_full, "speedup": ms_full / ms_part,
            "planted_weights_exact": exact}


def time_rows(tpd, L, torch, stream, n=14, seed=1005):
    """The remaining rows of the path, each timed on its own: zero skipping on
    the planted n=14 Heisenberg chain (dense storage, ~2^n(1+(n-1)/2)
    nonzeros), the composition (adjoint, scale 2^-n) of dense n=14 weights,
    and the autograd forward + backward at n=12 (L = sum w_t |c_t|^2)."""
    from paper_2310_13421_gb300 import synth
    out = {}
    J, h = synth.heisenberg_params(n, seed=seed)
    H = torch.from_numpy(synth.heisenberg(n, J, h)).cuda()
    work = torch.empty_like(H)
    wsb = L.tpd_workspace_size(n, L.TPD_C128, L.options(skip_zero=True))
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")

    def dec(skip):
        st = L.tpd_decompose(work.data_ptr(), n, L.TPD_C128, L.options(skip_zero=skip), ws.data_ptr(), wsb,
                             stream.cuda_stream)
        assert st == 0, L.status_string(st)

    ms_skip = _event_ms(torch, stream, lambda: dec(True), setup=lambda: work.copy_(H))
    ms_dense = _event_ms(torch, stream, lambda: dec(False), setup=lambda: work.copy_(H))
    out["zero_skip_heisenberg"] = {"skip_ms": ms_skip, "dense_ms": ms_dense, "speedup": ms_dense / ms_skip,
                                   "nonzeros": int(torch.count_nonzero(H).item())}
    # the same matrix from its nonzero entries (sparse input, Alg. 2 on entries)
    idx = torch.nonzero(H, as_tuple=True)
    rows, cols = idx[0].to(torch.int32).contiguous(), idx[1].to(torch.int32).contiguous()
    vals = H[idx].contiguous()
    nnz = vals.numel()
    max_entries = 4 * nnz + 1024
    wsp = torch.empty(L.tpd_sparse_workspace_size(max_entries), dtype=torch.uint8, device="cuda")
    strings = torch.empty(max_entries, dtype=torch.int64, device="cuda")
    weights = torch.empty(max_entries, dtype=torch.complex128, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    stat = torch.zeros(1, dtype=torch.int32, device="cuda")

    def sparse():
        st = L.tpd_decompose_coo(rows.data_ptr(), cols.data_ptr(), vals.data_ptr(), nnz, n, L.TPD_C128, max_entries,
                                 strings.data_ptr(), weights.data_ptr(), max_entries, cnt.data_ptr(), stat.data_ptr(),
                                 wsp.data_ptr(), wsp.numel(), stream.cuda_stream)
        assert st == 0, L.status_string(st)

    ms_sparse = _event_ms(torch, stream, sparse)
    terms = synth.heisenberg_terms(n, J, h)
    want = sorted(synth.string_index(t) for t in terms)
    k = int(cnt.item())
    out["sparse_coo_heisenberg"] = {"ms": ms_sparse, "nonzeros": nnz, "strings": k,
                                    "speedup_vs_dense": ms_dense / ms_sparse,
                                    "planted_strings_exact": int(stat.item()) == 0 and
                                    strings[:k].cpu().tolist() == want}
    del rows, cols, vals, wsp, strings, weights
    # composition with the adjoint scale on the weights of a dense matrix
    A = torch.from_numpy(synth.hermitian(n, seed=1002)).cuda()
    Wt = tpd.decompose(A)
    del A, H
    wsc = L.tpd_workspace_size(n, L.TPD_C128, L.options())
    wsc_t = torch.empty(max(wsc, 16), dtype=torch.uint8, device="cuda")

    def comp():
        st = L.tpd_compose(work.data_ptr(), n, L.TPD_C128, 2.0 ** -n, L.options(), wsc_t.data_ptr(), wsc,
                           stream.cuda_stream)
        assert st == 0, L.status_string(st)

    ms_comp = _event_ms(torch, stream, comp, setup=lambda: work.copy_(Wt))
    npass = L.tpd_plan_describe(n, L.TPD_C128, L.options())[0]
    out["compose_adjoint"] = {"ms": ms_comp, "passes": npass,
                              "hbm_gbs_per_pass": 2 * 16 * 4 ** n / (ms_comp / npass * 1e-3) / 1e9}
    del Wt, work
    torch.cuda.empty_cache()
    # autograd at n = 12: forward (decomposition) and backward (composition)
    m = 12
    A12 = torch.from_numpy(synth.hermitian(m, seed=1006)).cuda()
    wt = torch.rand(4 ** m, dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(1007)).view(2 ** m, 2 ** m)
    x = A12.clone().requires_grad_(True)

    def fwd_bwd():
        x.grad = None
        c = tpd.tpd(x)
        (wt * c.abs() ** 2).sum().backward()

    ms_ag = _event_ms(torch, stream, fwd_bwd)
    out["autograd_n12_fwd_bwd"] = {"ms": ms_ag, "note": "includes the torch loss and its gradient ops"}
    del A12, wt, x
    torch.cuda.empty_cache()
    return out


def time_helpers(tpd, L, torch, stream, n=14):
    """Memory-bound helpers on the n=14 complex128 matrix: RC -> string layout
    (read + write) and the fp64 sum of squares (read)."""
    from paper_2310_13421_gb300 import synth
    A = torch.from_numpy(synth.hermitian(n, seed=1002)).cuda()
    nbytes = A.numel() * 16
    S = torch.empty(A.numel(), dtype=A.dtype, device="cuda")
    code = L.TPD_C128

    def conv():
        st = L.tpd_convert_layout(A.data_ptr(), S.data_ptr(), n, code, 1, stream.cuda_stream)
        assert st == 0

    ms_layout = _event_ms(torch, stream, conv)
    ms_sumsq = _event_ms(torch, stream, lambda: tpd.sum_squares(A))
    del A, S
    torch.cuda.empty_cache()
    return {"layout_ms": ms_layout, "layout_gbs": 2 * nbytes / (ms_layout * 1e-3) / 1e9,
            "sum_squares_ms": ms_sumsq, "sum_squares_gbs": nbytes / (ms_sumsq * 1e-3) / 1e9}


# X-masks whose weights the accuracy leg compares with the oracle: all-I/Z,
# the extremes, and a fixed random sample
def accuracy_xs(n, count=16, seed=77):
    rng = np.random.default_rng(seed)
    base = [0, 1, 2 ** (n - 1), 2 ** n - 1]
    return np.array(base + [int(v) for v in rng.integers(1, 2 ** n, count - len(base))], dtype=np.int64)


def rows_of(W, n, xs):
    """The weights w_(x,z), z = 0..N-1, of each X-mask x in xs from a result
    W in RC layout (a CUDA tensor or a host array): row bits = z, column
    bits = x xor z."""
    z = np.arange(2 ** n, dtype=np.int64)
    pos = np.concatenate([((z << n) | (int(x) ^ z)) for x in xs])
    if hasattr(W, "is_cuda"):
        import torch
        got = W.reshape(-1).index_select(0, torch.from_numpy(pos).to(W.device)).cpu().numpy()
    else:
        got = np.asarray(W).reshape(-1)[pos]
    return got.astype(np.complex128).reshape(len(xs), 2 ** n)


def oracle_accuracy(A, n, xs, results):
    """Accuracy leg (CPU, after the timed regions, rank 0): each GPU result's
    error against the fp64 oracle on the sampled X-rows of the same input
    (a complex64 input widened exactly).  Reported per result: the normwise
    relative error over the sample; the largest error in units of
    m_x = 2^-n sum_r |A[r^x][r]| (the scale of fp64's componentwise bound);
    and the largest relative error among weights with |w| >= 1e-2 m_x."""
    import oracle
    want = oracle.coeffs_xrows(A, xs)
    r = np.arange(2 ** n, dtype=np.int64)
    m = np.array([np.abs(A[r ^ int(x), r].astype(np.complex128)).sum() / 2 ** n for x in xs])[:, None]
    out = {}
    for name, got in results.items():
        err = np.abs(got - want)
        big = np.abs(want) >= 1e-2 * m
        out[name] = {"normwise": float(np.linalg.norm(err) / np.linalg.norm(want)),
                     "max_over_m_x": float(np.max(err / m)),
                     "max_rel_above_1e-2_m_x": float(np.max(err[big] / np.abs(want[big]))),
                     "weights": int(want.size)}
    return out


def run_ours(args, world, rank, local):
    import torch
    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2310_13421_gb300 import dist as tdist

    def max_over_ranks(x):
        return tdist.max_over_ranks(x, device="cuda")

    import paper_2310_13421_gb300 as tpd
    from paper_2310_13421_gb300 import _lib as L, synth
    tpd.build()
    L.load()
    n = args.qubits
    N = 2 ** n
    coeffs = 4 ** n
    c64 = args.storage == "c64"
    elem = 8 if c64 else 16
    code = L.TPD_C64 if c64 else L.TPD_C128
    prec = {"default": L.TPD_PREC_DEFAULT, "fixed": L.TPD_PREC_FIXED, "plain": L.TPD_PREC_PLAIN,
            "compensated": L.TPD_PREC_COMPENSATED}[args.precision]
    prec_eff = prec if prec != L.TPD_PREC_DEFAULT else (L.TPD_PREC_PLAIN if c64 else L.TPD_PREC_FIXED)
    A = synth.hermitian(n, seed=SEED + rank, dtype=np.complex64 if c64 else np.complex128)
    A_pin = torch.from_numpy(A).pin_memory()
    pristine = A_pin.to("cuda", non_blocking=False)
    work = torch.empty_like(pristine)
    stream = torch.cuda.current_stream()

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    time.sleep(0.3)
    step_ms, pass_ms, npass = time_decompose(tpd, L, torch, work, pristine, n, args.steps, args.warmup,
                                             prec_eff, stream)
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(step_ms))
    ms_per_step = total_ms / args.steps
    value = tdist.job_rate(world * coeffs * args.steps, total_ms)

    # roofline of the pass kernel: algorithmic bytes per launch = read + write of the matrix
    alg_bytes = 2 * coeffs * elem
    launches = [ms for row in pass_ms for ms in row]
    mean_launch_ms = float(np.mean(launches))
    per_pass_ms = [float(np.mean([row[p] for row in pass_ms])) for p in range(npass)]
    achieved = alg_bytes / (mean_launch_ms * 1e-3) / 1e9
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if (c64 or prec_eff != L.TPD_PREC_FIXED) else measured_traffic(n),
                "kernel": ("k_pass_pf (first pass: persistent, prefetching) / k_pass<FixedArith,dec> "
                           "(later passes), compiled tile layouts; one launch per pass, %d passes" % npass)
                if (not c64 and prec_eff == L.TPD_PREC_FIXED) else
                "k_pass<%s,true> (one launch per pass, %d passes)" % (
                    {L.TPD_PREC_FIXED: "Fixed32Arith" if c64 else "FixedArith",
                     L.TPD_PREC_PLAIN: "F32Arith" if c64 else "F64Arith",
                     L.TPD_PREC_COMPENSATED: "F32CArith"}[prec_eff], npass),
                "bytes_per_launch": alg_bytes, "per_pass_ms": per_pass_ms,
                "per_pass_gbs": [alg_bytes / (m * 1e-3) / 1e9 for m in per_pass_ms],
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}

    # ---- end to end through the C ABI with pinned host buffers: every step
    # copies its input in and its result out (tpd_decompose_host); steps
    # alternate between two streams with their own device buffers, so one
    # step's device->host copy overlaps the next step's host->device copy
    # (the link is full duplex) -- the throughput a user gets from several streams
    ns_ = max(1, args.e2e_streams)
    W_pins = [torch.empty_like(A_pin).pin_memory() for _ in range(ns_)]
    works = [work] + [torch.empty_like(pristine) for _ in range(ns_ - 1)]
    streams = [stream] + [torch.cuda.Stream() for _ in range(ns_ - 1)]
    wsb = L.tpd_workspace_size(n, code, L.options(precision=prec_eff))
    wss = [torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda") for _ in range(ns_)]

    def e2e_step(k):
        j = k % ns_
        st = L.tpd_decompose_host(A_pin.data_ptr(), W_pins[j].data_ptr(), works[j].data_ptr(), n, code,
                                  L.options(precision=prec_eff), wss[j].data_ptr(), wsb, streams[j].cuda_stream)
        assert st == 0, L.status_string(st)

    for k in range(ns_):                    # warm-up, every stream
        e2e_step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(streams[0])
    for st_ in streams[1:]:
        st_.wait_event(e0)
    for k in range(args.e2e_steps):
        e2e_step(k)
    for st_ in streams[1:]:
        ej = torch.cuda.Event()
        ej.record(st_)
        streams[0].wait_event(ej)
    e1.record(streams[0])
    torch.cuda.synchronize()
    e2e_total = max_over_ranks(e0.elapsed_time(e1))
    e2e = {"value": tdist.job_rate(world * coeffs * args.e2e_steps, e2e_total), "unit": UNIT,
           "h2d_bytes_per_step": coeffs * elem, "d2h_bytes_per_step": coeffs * elem,
           "ms_per_step": e2e_total / args.e2e_steps, "steps": args.e2e_steps,
           "pipelining": "steps alternate over %d streams (own device buffers)" % ns_}
    # sanity: the host results equal the device results of the same plan
    ok = all(torch.equal(w.to("cuda"), d) for w, d in zip(W_pins, works))
    W_pin = W_pins[(args.e2e_steps - 1) % ns_]
    work = works[(args.e2e_steps - 1) % ns_]
    del works, wss, W_pins
    alg2 = None
    if rank == 0 and world == 1 and not args.no_extra and not c64:
        alg2 = alg2_baseline(A, W_pin.numpy(), n)

    extra = {}
    paper_arith = None
    acc_rows = {}            # results sampled for the accuracy leg: config -> (A, n, xs, {form: rows})
    weyl_rows = gm_rows = None
    if not args.no_extra and not c64 and prec_eff == L.TPD_PREC_FIXED:
        # fp64 butterfly (IEEE double, rounded per level) on the same matrix
        s64, p64, np64 = time_decompose(tpd, L, torch, work, pristine, n, 5, 2, L.TPD_PREC_PLAIN, stream)
        f64_ms = float(np.mean(s64))
        if rank == 0 and world == 1:
            xs14 = accuracy_xs(n)
            acc_rows["n%d_c128" % n] = (A, n, xs14, {"fixed": rows_of(W_pin.numpy(), n, xs14),
                                                    "fp64": rows_of(work, n, xs14)})
        extra["c128_fp64_plain_n%d" % n] = {"ms_per_step": f64_ms, "coeffs_per_s": coeffs / (f64_ms * 1e-3),
                                        "passes": np64}
        # the same metric in the paper's arithmetic (IEEE fp64 adds rounded
        # every level), reported beside the default block fixed point
        f64_pass = [float(np.mean([row[p] for row in p64])) for p in range(np64)]
        f64_achieved = alg_bytes / (float(np.mean(f64_pass)) * 1e-3) / 1e9
        paper_arith = {"label": "paper arithmetic: IEEE fp64 adds rounded after every level",
                       "value": tdist.job_rate(world * coeffs * len(s64), max_over_ranks(sum(s64))), "unit": UNIT,
                       "ms_per_step": f64_ms, "dtype": "f64", "passes": np64,
                       "roofline": {"bound": "hbm", "achieved": f64_achieved, "peak": peak, "unit": "GB/s",
                                    "frac": f64_achieved / peak, "kernel": "k_pass<F64Arith,true>",
                                    "per_pass_ms": f64_pass,
                                    "note": "fp64-add bound on GB300 (its fp64 pipe), not HBM bound"}}
        extra["c128_fixed_n%d" % n] = {"ms_per_step": ms_per_step, "coeffs_per_s": coeffs / (ms_per_step * 1e-3)}
        del work, pristine
        torch.cuda.empty_cache()
        # complex64 at n = 15: plain and compensated fp32 vs fp64 / fixed complex128 of the same matrix
        n15 = 15
        A64 = synth.hermitian(n15, seed=1003, dtype=np.complex64)
        p15 = torch.from_numpy(A64).cuda()
        w15 = torch.empty_like(p15)
        res = {}
        for name, prec in (("plain", L.TPD_PREC_PLAIN), ("compensated", L.TPD_PREC_COMPENSATED),
                           ("fixed", L.TPD_PREC_FIXED)):
            s, _, npp = time_decompose(tpd, L, torch, w15, p15, n15, 5, 2, prec, stream)
            res[name] = {"ms_per_step": float(np.mean(s)), "coeffs_per_s": 4 ** n15 / (np.mean(s) * 1e-3),
                         "passes": npp, "hbm_gbs_per_pass": 2 * 4 ** n15 * 8 / (np.mean(s) / npp * 1e-3) / 1e9}
            res[name]["_out"] = w15.clone()
        ref = tpd.decompose(p15.to(torch.complex128), precision="fixed")
        xs15 = accuracy_xs(n15)
        rows15 = {}
        for name in ("plain", "compensated", "fixed"):
            out = res[name].pop("_out")
            rows15["c64_" + name] = rows_of(out, n15, xs15)
            out = out.to(torch.complex128)
            res[name]["rel_err_vs_c128"] = float(torch.linalg.vector_norm(out - ref) / torch.linalg.vector_norm(ref))
            del out
        del ref
        w128 = p15.to(torch.complex128)
        p128 = w128.clone()
        s, _, npp = time_decompose(tpd, L, torch, w128, p128, n15, 3, 1, L.TPD_PREC_PLAIN, stream)
        res["c128_fp64_plain"] = {"ms_per_step": float(np.mean(s)), "passes": npp}
        rows15["c128_fp64"] = rows_of(w128, n15, xs15)
        s, _, npp = time_decompose(tpd, L, torch, w128, p128, n15, 3, 1, L.TPD_PREC_FIXED, stream)
        res["c128_fixed"] = {"ms_per_step": float(np.mean(s)), "passes": npp}
        rows15["c128_fixed"] = rows_of(w128, n15, xs15)
        if rank == 0 and world == 1:
            acc_rows["n15_c64_input"] = (A64, n15, xs15, rows15)
        extra["n15"] = res
        extra["speedup_c64_compensated_vs_c128_fp64_n15"] = res["c128_fp64_plain"]["ms_per_step"] / \
            res["compensated"]["ms_per_step"]
        extra["speedup_c64_compensated_vs_c128_fixed_n15"] = res["c128_fixed"]["ms_per_step"] / \
            res["compensated"]["ms_per_step"]
        extra["speedup_c64_fixed_vs_c128_fp64_n15"] = res["c128_fp64_plain"]["ms_per_step"] / \
            res["fixed"]["ms_per_step"]
        del w128, p128, p15, w15
        torch.cuda.empty_cache()
        extra["partial_n14_heisenberg"] = time_partial(tpd, L, torch, stream)
        extra["rows_n14"] = time_rows(tpd, L, torch, stream)
        extra["helpers_n14"] = time_helpers(tpd, L, torch, stream)
        extra["weyl_d3_n9"], weyl_rows = time_weyl(tpd, L, torch, stream)
        extra["gellmann_d3_n9"], gm_rows = time_gellmann(tpd, L, torch, stream, A=weyl_rows[0])
    if not args.no_extra and not args.no_batch and not c64:
        extra["batch_4096_n3_10"] = time_batch(tpd, L, torch, stream)

    cpu = None
    if rank == 0 and world == 1:
        v, cores, sample = oracle_rate(A, n)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    if alg2 is not None:
        extra["cpu_alg2_1thread"] = alg2["alg2_1thread"]
        extra["cpu_alg2"] = alg2["alg2"]
    if acc_rows:
        extra["error_vs_fp64_oracle"] = {cfg: oracle_accuracy(*v) for cfg, v in acc_rows.items()}
        acc_rows.clear()
    if weyl_rows is not None and rank == 0 and world == 1:
        extra["weyl_d3_n9"]["error_vs_fp64_oracle"] = weyl_accuracy(*weyl_rows)
        weyl_rows = None
    if gm_rows is not None and rank == 0 and world == 1:
        extra["gellmann_d3_n9"]["error_vs_fp64_oracle"] = gellmann_accuracy(*gm_rows)
        gm_rows = None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {L.TPD_PREC_FIXED: "int64", L.TPD_PREC_PLAIN: "f32" if c64 else "f64",
                                       L.TPD_PREC_COMPENSATED: "f32"}[prec_eff], "data": "synthetic",
        "config": {"workload": "n=%d dense random Hermitian, %dx%d " % (n, N, N) +
                               ("complex64" if c64 else "complex128") +
                               " (%.2f GB) in place; Re,Im of B ~ N(0,1), A=(B+B^H)/2" % (coeffs * elem / 1e9),
                   "storage": "complex64" if c64 else "complex128",
                   "precision": {L.TPD_PREC_FIXED: "fixed: int64 block fixed point, one binary point per "
                                                   "class of summed elements, one rounding per pass",
                                 L.TPD_PREC_PLAIN: "plain IEEE adds per level",
                                 L.TPD_PREC_COMPENSATED: "compensated fp32 (TwoSum per pass)"}[prec_eff],
                   "passes": npass,
                   "l2": "inputs larger than L2 (%.2f GB vs 126 MB); restored between steps" % (coeffs * elem / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "clocks": clk, "gpu_launches": args.steps * npass,
        "e2e_matches_device": bool(ok), "extra": extra,
    }
    if paper_arith is not None:
        line["paper_arithmetic"] = paper_arith
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch_only(args):
    import torch
    import paper_2310_13421_gb300 as tpd
    from paper_2310_13421_gb300 import _lib as L
    tpd.build()
    L.load()
    res = time_batch(tpd, L, torch, torch.cuda.current_stream(), count=args.batch_count, reps=args.steps)
    print(json.dumps({"workload": "batch of %d complex128 Hermitian matrices, n ~ U{3..10}" % args.batch_count,
                      "batch": res}))
    return 0


def run_weyl_only(args):
    import torch
    import paper_2310_13421_gb300 as tpd
    from paper_2310_13421_gb300 import _lib as L
    tpd.build()
    L.load()
    res, rows = time_weyl(tpd, L, torch, torch.cuda.current_stream(), n=args.weyl_n)
    res["error_vs_fp64_oracle"] = weyl_accuracy(*rows)
    print(json.dumps({"workload": "Weyl basis, d = 3, n = %d" % args.weyl_n, "weyl": res}))
    return 0


def run_gellmann_only(args):
    import torch
    import paper_2310_13421_gb300 as tpd
    from paper_2310_13421_gb300 import _lib as L
    tpd.build()
    L.load()
    res, rows = time_gellmann(tpd, L, torch, torch.cuda.current_stream(), n=args.weyl_n)
    res["error_vs_fp64_oracle"] = gellmann_accuracy(*rows)
    print(json.dumps({"workload": "generalized Gell-Mann basis, d = 3, n = %d" % args.weyl_n, "gellmann": res}))
    return 0


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "batch":
        return run_batch_only(args)
    if args.workload == "weyl":
        return run_weyl_only(args)
    if args.workload == "gellmann":
        return run_gellmann_only(args)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
