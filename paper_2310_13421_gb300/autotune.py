"""Autotuner for the pass plans.

For a (qubits n, storage dtype, precision) key it times candidate tunings --
the tile size (``tile_bits``, elements per CTA tile), the most levels fused in
one pass (``max_levels``) and the kernel form (``variant``: per-tile CTAs at
the planner's occupancy or forced to 2 / 3 CTAs per SM, or the persistent
prefetching form) -- on the current GPU with CUDA events, keeps only
candidates that reproduce the default plan's result exactly on an integer
input, registers the fastest with ``tpd_tune_set`` (so single and batched
calls use it) and caches the choice in a JSON file keyed by GPU name and SM
count.  Small n is tuned on a batch of matrices through the batched call.
``tune_batch`` tunes for a given mixed batch instead: every qubit count inside
the batch it serves, timed as the whole batch, never slower than the
planner's defaults on it.
"""
import itertools
import json
import os

import torch

from . import _lib as L
from . import synth

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "tpd_autotune.json")

_DT = {"c128": (L.TPD_C128, torch.complex128), "c64": (L.TPD_C64, torch.complex64)}
_PREC = {"default": L.TPD_PREC_DEFAULT, "plain": L.TPD_PREC_PLAIN, "compensated": L.TPD_PREC_COMPENSATED,
         "fixed": L.TPD_PREC_FIXED}


def _gpu_key():
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def candidates(n, dtype, precision, batched=False):
    """Distinct valid tunings for the key (same plan text and variant = same
    candidate).  For batches, variant 2 (one persistent launch for the whole
    batch) competes with the default launch per qubit count and pass."""
    code = _DT[dtype][0]
    prec = _PREC[precision] if isinstance(precision, str) else precision
    seen, out = set(), []
    variants = (0, 2, 3, 4)
    for tb, ml, var in itertools.product((0, 11, 12, 13), (0, 3, 4, 5, 6), variants):
        opt = L.options(precision=prec, tile_bits=tb, max_levels=ml, variant=var)
        npass, desc = L.tpd_plan_describe(n, code, opt)
        if npass < 0:
            continue
        if var == 2 and not batched and (code != L.TPD_C128 or npass == 0):
            continue          # single matrices: the persistent form exists for the complex128 fixed point
        key = (desc, var)
        if key in seen:
            continue
        seen.add(key)
        out.append(dict(tile_bits=tb, max_levels=ml, variant=var, passes=npass))
    return out


def _time_single(n, code, tdt, prec, cand, reps):
    A = torch.from_numpy(synth.hermitian(n, seed=77)).to("cuda", tdt)
    W = torch.empty_like(A)
    opt = L.options(precision=prec, tile_bits=cand["tile_bits"], max_levels=cand["max_levels"],
                    variant=cand["variant"])
    wsb = L.tpd_workspace_size(n, code, opt)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    times = []
    for k in range(reps + 2):
        W.copy_(A)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = L.tpd_decompose(W.data_ptr(), n, code, opt, ws.data_ptr(), wsb, s.cuda_stream)
        e1.record(s)
        if st != L.TPD_OK:
            return None
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def _time_batch(n, code, tdt, prec, cand, reps, count):
    mats = [torch.from_numpy(synth.hermitian(n, seed=1000 + i)).to("cuda", tdt) for i in range(count)]
    orig = [m.clone() for m in mats]
    opt = L.options(precision=prec, tile_bits=cand["tile_bits"], max_levels=cand["max_levels"],
                    variant=cand["variant"])
    ptrs = torch.tensor([m.data_ptr() for m in mats], dtype=torch.int64, device="cuda")
    ns = [n] * count
    ns_dev = torch.tensor(ns, dtype=torch.int32, device="cuda")
    wsb = L.tpd_batched_workspace_size(ns, code, opt)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    times = []
    for k in range(reps + 2):
        for m, o in zip(mats, orig):
            m.copy_(o)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = L.tpd_decompose_batched(ptrs.data_ptr(), ns_dev.data_ptr(), ns, code, opt, ws.data_ptr(), wsb,
                                     s.cuda_stream)
        e1.record(s)
        if st != L.TPD_OK:
            return None
        torch.cuda.synchronize()
        if k >= 2:
            times.append(e0.elapsed_time(e1))
    times.sort()
    return times[len(times) // 2]


def _agrees_with_default(n, code, tdt, prec, cand):
    """The candidate reproduces the default plan bit for bit on an integer input."""
    A = torch.from_numpy(synth.int_general(min(n, 10), seed=5)).to("cuda", tdt)
    m = A.shape[0].bit_length() - 1
    outs = []
    for c in (dict(tile_bits=0, max_levels=0, variant=1), cand):
        W = A.clone()
        opt = L.options(precision=prec, tile_bits=c["tile_bits"], max_levels=c["max_levels"], variant=c["variant"])
        if L.tpd_plan_describe(m, code, opt)[0] < 0:
            return True       # the candidate has no plan at the check size; timed size decides
        wsb = L.tpd_workspace_size(m, code, opt)
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
        if L.tpd_decompose(W.data_ptr(), m, code, opt, ws.data_ptr(), wsb,
                           torch.cuda.current_stream().cuda_stream) != L.TPD_OK:
            return False
        outs.append(W)
    torch.cuda.synchronize()
    return bool(torch.equal(outs[0], outs[1]))


def tune(n, dtype="c128", precision="default", reps=5, batch_bytes=64 << 20, register=True, cache=None):
    """Time every candidate for (n, dtype, precision); register and cache the
    fastest.  Returns {"best": {...}, "ms": t, "default_ms": t0, "tried": [...]}."""
    code, tdt = _DT[dtype]
    prec = _PREC[precision] if isinstance(precision, str) else precision
    L.tpd_tune_set(n, code, prec, None)          # time against the planner, not an old choice
    elem = 16 if dtype == "c128" else 8
    count = max(1, batch_bytes // (4 ** n * elem)) if n <= 10 else 1
    tried = []
    for cand in candidates(n, dtype, prec, batched=count > 1):
        if not _agrees_with_default(n, code, tdt, prec, cand):
            continue
        t = _time_batch(n, code, tdt, prec, cand, reps, count) if count > 1 else \
            _time_single(n, code, tdt, prec, cand, reps)
        if t is not None:
            tried.append(dict(cand, ms=t))
    if not tried:
        raise RuntimeError("no candidate ran for n=%d %s" % (n, dtype))
    default = [c for c in tried if c["tile_bits"] == 0 and c["max_levels"] == 0 and c["variant"] == 0]
    best = min(tried, key=lambda c: c["ms"])
    res = {"best": {k: best[k] for k in ("tile_bits", "max_levels", "variant")}, "ms": best["ms"],
           "default_ms": default[0]["ms"] if default else None, "batch": count, "tried": tried}
    if register:
        L.tpd_tune_set(n, code, prec, L.options(precision=prec, **res["best"]))
    if cache is not None:
        save(cache, n, dtype, prec, res)
    return res


def tune_batch(mats, precision="default", reps=3, margin=0.01, register=True):
    """Tune for the batch the choices will serve: `mats`, CUDA matrices of
    mixed sizes (all complex128 or all complex64), decomposed in place by the
    batched call.  Starting from the planner's defaults, each qubit count in
    the batch in turn tries its candidates (tile bits, levels per pass, CTAs
    per SM) with the others fixed, timing the WHOLE batch; a candidate
    replaces the incumbent only when the batch runs faster by more than
    `margin`.  Finally the batch-wide form -- one launch per (qubit count,
    pass) or one persistent launch -- is chosen the same way.  The defaults
    are the first incumbents, so the result is never slower than them on this
    batch (up to timing noise).  The matrices are restored after every run.
    Returns {"per_n": {n: choice}, "variant": 0 or 2, "ms": t, "default_ms": t0}."""
    if not mats:
        raise ValueError("empty batch")
    code, tdt = (L.TPD_C128, torch.complex128) if mats[0].dtype == torch.complex128 else (L.TPD_C64, torch.complex64)
    prec = _PREC[precision] if isinstance(precision, str) else precision
    ns = [m.shape[0].bit_length() - 1 for m in mats]
    orig = [m.clone() for m in mats]
    ptrs = torch.tensor([m.data_ptr() for m in mats], dtype=torch.int64, device="cuda")
    ns_dev = torch.tensor(ns, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    for n in set(ns):
        L.tpd_tune_set(n, code, prec, None)
    choice = {n: dict(tile_bits=0, max_levels=0, variant=0) for n in set(ns)}

    def run(batch_variant):
        opt = L.options(precision=prec, variant=batch_variant)
        wsb = L.tpd_batched_workspace_size(ns, code, opt)
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
        times = []
        for k in range(reps + 2):
            for m, o in zip(mats, orig):
                m.copy_(o)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            st = L.tpd_decompose_batched(ptrs.data_ptr(), ns_dev.data_ptr(), ns, code, opt, ws.data_ptr(), wsb,
                                         s.cuda_stream)
            e1.record(s)
            if st != L.TPD_OK:
                return None
            torch.cuda.synchronize()
            if k >= 2:
                times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2]

    def apply(n, c):
        if c["tile_bits"] == 0 and c["max_levels"] == 0 and c["variant"] == 0:
            return L.tpd_tune_set(n, code, prec, None) == L.TPD_OK
        return L.tpd_tune_set(n, code, prec, L.options(precision=prec, **c)) == L.TPD_OK

    default_ms = best_ms = run(0)
    for n in sorted(set(ns), key=lambda k: -ns.count(k) * 4 ** k):     # the largest share of the work first
        for cand in candidates(n, "c128" if code == L.TPD_C128 else "c64", prec, batched=True):
            c = {k: cand[k] for k in ("tile_bits", "max_levels", "variant")}
            if c == choice[n] or c["variant"] == 2:       # the batch-wide form is chosen below
                continue
            if not _agrees_with_default(n, code, tdt, prec, cand) or not apply(n, c):
                apply(n, choice[n])
                continue
            t = run(0)
            if t is not None and t < best_ms * (1.0 - margin):
                best_ms, choice[n] = t, c
            else:
                apply(n, choice[n])
    batch_variant = 0
    t2 = run(2)
    if t2 is not None and t2 < best_ms * (1.0 - margin):
        best_ms, batch_variant = t2, 2
    for m, o in zip(mats, orig):
        m.copy_(o)
    if not register:
        for n in set(ns):
            L.tpd_tune_set(n, code, prec, None)
    return {"per_n": choice, "variant": batch_variant, "ms": best_ms, "default_ms": default_ms}


def save(path, n, dtype, precision, res):
    data = {}
    if os.path.exists(path):
        with open(path) as fh:
            data = json.load(fh)
    data.setdefault(_gpu_key(), {})["%d/%s/%d" % (n, dtype, precision)] = {
        "best": res["best"], "ms": res["ms"], "default_ms": res["default_ms"]}
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def load(path=None):
    """Register the cached choices for this GPU; returns how many."""
    path = path or os.environ.get("TPD_AUTOTUNE_CACHE", DEFAULT_CACHE)
    if not os.path.exists(path):
        return 0
    with open(path) as fh:
        entries = json.load(fh).get(_gpu_key(), {})
    k = 0
    for key, val in entries.items():
        n, dtype, prec = key.split("/")
        code = _DT[dtype][0]
        if L.tpd_tune_set(int(n), code, int(prec), L.options(precision=int(prec), **val["best"])) == L.TPD_OK:
            k += 1
    return k
