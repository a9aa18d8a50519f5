"""Host-side tests of libtpd.so (no GPU needed): the library loads, exports
every symbol include/tpd.h declares, rejects bad arguments before touching the
device, and its pass plans are valid -- checked by emulating each plan's data
movement on the CPU and comparing with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2310_13421_gb300 import buildlib, _lib
    buildlib.build()
    _lib.load()
    return _lib


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "tpd.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpd_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    lib = ctypes.CDLL(L.LIB)
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(L.SYMBOLS)


def test_status_strings_and_version(L):
    assert L.status_string(0) == "TPD_OK"
    assert L.status_string(6) == "TPD_ERR_TIMEOUT"
    assert L.tpd_version() >= 100


def test_argument_errors_return_before_any_launch(L):
    # none of these reaches the CUDA runtime
    assert L.tpd_decompose(0, 4, L.TPD_C128) == L.TPD_ERR_INVALID_ARG          # null
    assert L.tpd_decompose(4096, 0, L.TPD_C128) == L.TPD_ERR_INVALID_ARG       # n = 0
    assert L.tpd_decompose(4096, 17, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # n too big
    assert L.tpd_decompose(4096, 4, 7) == L.TPD_ERR_INVALID_ARG                # dtype
    assert L.tpd_decompose(4104, 4, L.TPD_C128) == L.TPD_ERR_MISALIGNED        # 8 mod 16
    assert L.tpd_decompose(4100, 4, L.TPD_C64) == L.TPD_ERR_MISALIGNED         # 4 mod 8
    assert L.tpd_decompose(4096, 4, L.TPD_C128, L.options(precision=2)) == L.TPD_ERR_UNSUPPORTED
    assert L.tpd_plan_describe(12, L.TPD_C64, L.options(precision=3))[0] >= 2        # complex64 fixed point
    assert L.tpd_decompose(4096, 4, L.TPD_C128, L.options(precision=9)) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_decompose(4096, 4, L.TPD_C128, L.options(tile_bits=20)) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_compose(4096, 8, L.TPD_C128, 0.0) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_compose(4096, 8, L.TPD_C128, float("inf")) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_compose(4096, 3, L.TPD_C128, 3.0) == L.TPD_ERR_UNSUPPORTED   # whole-matrix: 1 or 2^-n
    # zero skip on a multi-pass plan needs the workspace
    assert L.tpd_workspace_size(10, L.TPD_C128, L.options(precision=1, skip_zero=True)) > 0
    assert L.tpd_workspace_size(10, L.TPD_C128, L.options(precision=1)) == 0
    assert L.tpd_decompose(4096, 10, L.TPD_C128, L.options(precision=1, skip_zero=True)) == L.TPD_ERR_WORKSPACE
    # the block fixed point hands one int16 binary point per class (4^n / 2^K
    # of them for a pass of K levels) to the next pass: n = 14, passes of 6, 4
    # and 4 levels, 2 x 2^22 + 2 x 2^24 bytes; zero skipping adds one flag
    # byte per tile of the passes after the first (the middle pass on
    # 2^11-element tiles, 2^17 of them; the last on 2^12, 2^16)
    ws = L.tpd_workspace_size(14, L.TPD_C128, L.options())
    assert ws == 2 * 2 ** 22 + 2 * 2 ** 24
    assert L.tpd_workspace_size(14, L.TPD_C128, L.options(skip_zero=True)) == ws + 2 ** 17 + 2 ** 16
    assert L.tpd_workspace_size(14, L.TPD_C128, L.options(precision=1)) == 0      # IEEE: nothing handed on
    assert L.tpd_workspace_size(6, L.TPD_C128, L.options(skip_zero=True)) == 0    # one pass: nothing to hand on
    assert L.tpd_decompose(4096, 10, L.TPD_C128) == L.TPD_ERR_WORKSPACE
    assert L.tpd_decompose(4096, 10, L.TPD_C128, None, 4104, 1 << 20) == L.TPD_ERR_MISALIGNED
    # batched
    assert L.tpd_batched_workspace_size([3, 4, 13], L.TPD_C128) == 0
    assert L.tpd_batched_workspace_size([3, 4, 10], L.TPD_C128) > 0
    assert L.tpd_decompose_batched(0, 0, [3, 4], L.TPD_C128) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_decompose_batched(4096, 4096, [3, 0], L.TPD_C128, None, 4096, 1 << 20) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_decompose_batched(4096, 4096, [3, 4], L.TPD_C128, None, 0, 0) == L.TPD_ERR_WORKSPACE
    assert L.tpd_decompose_batched(4096, 4096, [3, 4], L.TPD_C128, L.options(skip_zero=True), 4096,
                                   1 << 20) == L.TPD_ERR_UNSUPPORTED
    assert L.tpd_batch_status(0) == L.TPD_ERR_INVALID_ARG
    # partial decomposition
    assert L.tpd_partial_workspace_size(10, L.TPD_C128, None, 5) >= 5 * 8 + 2 * 256
    assert L.tpd_partial_workspace_size(10, L.TPD_C128, L.options(skip_zero=True), 5) == 0
    assert L.tpd_partial_prepare(4, L.TPD_C128, None, [1, 2], 0, 0) == L.TPD_ERR_WORKSPACE
    assert L.tpd_partial_prepare(4, L.TPD_C128, None, [256], 4096, 1 << 20) == L.TPD_ERR_INVALID_ARG  # >= 4^n
    assert L.tpd_decompose_partial(0, 4, L.TPD_C128, None, 2, 4096, 1 << 20, 8192) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_decompose_partial(4096, 4, L.TPD_C128, None, 2, 4096, 1 << 20, 8200) == L.TPD_ERR_MISALIGNED
    # sparse input
    assert L.tpd_sparse_workspace_size(1000) > 1000 * 40
    assert L.tpd_decompose_coo(4096, 4096, 4096, 1, 16, L.TPD_C128, 10, 0, 0, 0, 8192, 0, 1 << 20, 1 << 20) == \
        L.TPD_ERR_INVALID_ARG
    assert L.tpd_decompose_coo(4096, 4096, 4096, 1, 8, L.TPD_C64, 10, 0, 0, 0, 8192, 0, 1 << 20, 1 << 20) == \
        L.TPD_ERR_UNSUPPORTED
    assert L.tpd_decompose_coo(4096, 4096, 4096, 1, 8, L.TPD_C128, 10, 0, 0, 0, 8192, 0, 0, 0) == L.TPD_ERR_WORKSPACE
    # nonzero list
    assert L.tpd_nonzero_workspace_size(0) == 0 and L.tpd_nonzero_workspace_size(14) > 4 ** 10 * 4
    assert L.tpd_nonzero_list(4096, 4, L.TPD_C128, 0.0, 0, 0, 0, 8192, 0, 0) == L.TPD_ERR_WORKSPACE
    assert L.tpd_nonzero_list(4096, 4, L.TPD_C128, -1.0, 0, 0, 0, 8192, 1 << 20, 4096) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_nonzero_list(4096, 4, L.TPD_C128, 0.0, 0, 0, 5, 8192, 1 << 20, 4096) == L.TPD_ERR_INVALID_ARG
    # Weyl basis: d in 2..5, d^n <= 65536
    assert L.tpd_weyl_decompose(4096, 3, 1, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # d = 1
    assert L.tpd_weyl_decompose(4096, 3, 6, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # d = 6
    assert L.tpd_weyl_decompose(4096, 0, 3, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # n = 0
    assert L.tpd_weyl_decompose(4096, 11, 3, L.TPD_C128) == L.TPD_ERR_INVALID_ARG     # 3^11 > 65536
    assert L.tpd_weyl_decompose(0, 3, 3, L.TPD_C128) == L.TPD_ERR_INVALID_ARG         # null
    assert L.tpd_weyl_decompose(4096, 3, 3, 5) == L.TPD_ERR_INVALID_ARG               # dtype
    assert L.tpd_weyl_decompose(4104, 3, 3, L.TPD_C128) == L.TPD_ERR_MISALIGNED
    assert L.tpd_weyl_compose(4096, 3, 3, L.TPD_C128, 0.0) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_weyl_compose(4100, 3, 3, L.TPD_C64, 1.0) == L.TPD_ERR_MISALIGNED
    fixed, comp = L.options(precision=L.TPD_PREC_FIXED), L.options(precision=L.TPD_PREC_COMPENSATED)
    assert L.tpd_weyl_decompose(4096, 3, 3, L.TPD_C64, fixed) == L.TPD_ERR_INVALID_ARG      # fixed: complex128
    assert L.tpd_weyl_decompose(4096, 3, 5, L.TPD_C128, fixed) == L.TPD_ERR_INVALID_ARG     # fixed: d <= 4
    assert L.tpd_weyl_decompose(4096, 3, 3, L.TPD_C128, comp) == L.TPD_ERR_INVALID_ARG      # no compensated form
    # generalized Gell-Mann basis: d in 2..5, d^n <= 65536, IEEE arithmetic only
    assert L.tpd_gellmann_decompose(4096, 3, 1, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # d = 1
    assert L.tpd_gellmann_decompose(4096, 3, 6, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # d = 6
    assert L.tpd_gellmann_decompose(4096, 0, 3, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # n = 0
    assert L.tpd_gellmann_decompose(4096, 7, 5, L.TPD_C128) == L.TPD_ERR_INVALID_ARG      # 5^7 > 65536
    assert L.tpd_gellmann_decompose(0, 3, 3, L.TPD_C128) == L.TPD_ERR_INVALID_ARG         # null
    assert L.tpd_gellmann_decompose(4096, 3, 3, 5) == L.TPD_ERR_INVALID_ARG               # dtype
    assert L.tpd_gellmann_decompose(4104, 3, 3, L.TPD_C128) == L.TPD_ERR_MISALIGNED
    assert L.tpd_gellmann_decompose(4096, 3, 3, L.TPD_C128, fixed) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_gellmann_decompose(4096, 3, 3, L.TPD_C64, comp) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_gellmann_compose(4096, 3, 3, L.TPD_C128, 0.0) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_gellmann_compose(4096, 3, 3, L.TPD_C128, float("inf")) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_gellmann_compose(4100, 3, 3, L.TPD_C64, 1.0) == L.TPD_ERR_MISALIGNED
    # layout conversion and sums of squares
    assert L.tpd_convert_layout(4096, 1 << 20, 0, L.TPD_C128, 1) == L.TPD_ERR_INVALID_ARG      # n = 0
    assert L.tpd_convert_layout(4096, 4096 + 256, 4, L.TPD_C128, 1) == L.TPD_ERR_INVALID_ARG   # overlap
    assert L.tpd_convert_layout(4104, 1 << 20, 4, L.TPD_C128, 1) == L.TPD_ERR_MISALIGNED
    assert L.tpd_convert_layout(4096, 1 << 20, 4, L.TPD_C128, 2) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_sum_squares(4096, 10, L.TPD_C128, 8192, 0, 0) == L.TPD_ERR_WORKSPACE
    assert L.tpd_sum_squares(4096, 10, L.TPD_C128, 0, 1 << 20, 8192) == L.TPD_ERR_INVALID_ARG
    assert L.tpd_sum_squares(4104, 10, L.TPD_C128, 8192, 1 << 20, 8192) == L.TPD_ERR_MISALIGNED
    # workspace: control words (status, work counter, one completion counter per
    # matrix and pass but the last) + bucket list + bucketed pointers
    base = L.tpd_batched_workspace_size([3, 5], L.TPD_C128)
    assert base % 256 == 0 and base >= 256 + 256
    two_pass = L.tpd_batched_workspace_size([10] * 100, L.TPD_C128)
    assert two_pass >= 4 * (4 + 100) + 4 * 100 + 8 * 100 + 2 * 100 * 4 ** 10 // 2 ** 6


# ------------------------------------------------------------------ plan emulation

def _parse(desc):
    passes = []
    for line in desc.strip().splitlines():
        if not line.startswith("pass "):
            continue
        head, *stages = line.split(" | ")
        m = re.match(r"pass \d+: levels \[(\d+),(\d+)\) D=(\d+) tiles=(\d+) ctas=(\d+) gbits=([\d,]+)", head)
        b, e, D, ntiles, ctas, gbits = m.groups()
        p = dict(b=int(b), K=int(e) - int(b), D=int(D), ntiles=int(ntiles), ctas=int(ctas),
                 gbits=[int(x) for x in gbits.split(",")], stages=[])
        for st in stages:
            kv = dict(re.findall(r"(\w+)=([\d,]*)", st))
            ints = lambda k: [int(x) for x in kv[k].split(",")] if kv.get(k) else []
            p["stages"].append(dict(npair=int(kv["pairs"]), nshfl=int(kv["shfl"]), reg=ints("reg"),
                                    lane=ints("lane"), warp=ints("warp"), shfl_lane=ints("shfl_lane")))
        passes.append(p)
    return passes


def _level_on(x, cpos, rpos, dec=True):
    """Eq. 4 applied to tile axis pair (column bit cpos, row bit rpos) of x[..., 2^D]."""
    D = x.shape[-1].bit_length() - 1
    shp = [2] * D
    y = x.reshape(shp[::-1])  # numpy axis k <-> tile bit D-1-k
    ac, ar = D - 1 - cpos, D - 1 - rpos

    def sl(r, c):
        idx = [slice(None)] * D
        idx[ar], idx[ac] = r, c
        return tuple(idx)

    a00, a01, a10, a11 = (y[sl(0, 0)].copy(), y[sl(0, 1)].copy(), y[sl(1, 0)].copy(), y[sl(1, 1)].copy())
    y[sl(0, 0)] = (a00 + a11) / 2
    y[sl(0, 1)] = (a01 + a10) / 2
    y[sl(1, 0)] = 1j * (a01 - a10) / 2
    y[sl(1, 1)] = (a00 - a11) / 2
    return y.reshape(-1)


def _emulate(A, passes, n):
    flat = A.reshape(-1).copy()
    for p in passes:
        D, gb = p["D"], p["gbits"]
        rest = [g for g in range(2 * n) if g not in gb]
        tidx = np.arange(1 << D)
        off_in = np.zeros(1 << D, dtype=np.int64)
        for i, g in enumerate(gb):
            off_in += ((tidx >> i) & 1) << g
        for tile in range(p["ntiles"]):
            base = sum(((tile >> j) & 1) << g for j, g in enumerate(rest))
            x = flat[base + off_in]
            done = []
            for st in p["stages"]:
                # every stage mapping must be a bijection of the D tile bits
                assert sorted(st["reg"] + st["lane"] + st["warp"]) == list(range(D))
                assert set(range(3)) <= set(st["lane"])
                lv = []
                for q in range(st["npair"]):
                    lv.append((st["reg"][2 * q], st["reg"][2 * q + 1]))
                for s in range(st["nshfl"]):
                    lv.append((st["lane"][st["shfl_lane"][s]], st["reg"][2 * st["npair"] + s]))
                for cpos, rpos in lv:
                    # the pair must be one level's column and row bit
                    c, r = gb[cpos], gb[rpos]
                    assert r == c + n and p["b"] <= c < p["b"] + p["K"]
                    x = _level_on(x, cpos, rpos)
                    done.append(c)
            assert sorted(done) == list(range(p["b"], p["b"] + p["K"]))
            flat[base + off_in] = x
    return flat


def _to_string_order(flat, n):
    # independent of the package helper: walk strings, place t_j = 2 r + c
    out = np.empty(4 ** n, dtype=flat.dtype)
    N = 1 << n
    for s in range(4 ** n):
        r = c = 0
        for beta in range(n):
            t = (s >> (2 * beta)) & 3
            r |= (t >> 1) << beta
            c |= (t & 1) << beta
        out[s] = flat[r * N + c]
    return out


def _min_tile_bits(L):
    # register bits of a thread (one stage's register list) plus five lane bits
    return len(_parse(L.tpd_plan_describe(14, 0, L.options())[1])[0]["stages"][0]["reg"]) + 5


@pytest.mark.parametrize("n,dtype,prec", [(4, 0, 0), (4, 1, 2), (5, 0, 0), (6, 0, 0), (7, 0, 0), (8, 0, 0),
                                          (7, 1, 0), (8, 1, 2), (9, 0, 0), (9, 1, 3)])
def test_plans_emulated_on_cpu_match_oracle(L, n, dtype, prec):
    npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec))
    if 2 * n < _min_tile_bits(L):
        assert npass == 0                     # the single-CTA small path
        return
    passes = _parse(desc)
    assert len(passes) == npass
    assert sum(p["K"] for p in passes) == n
    A = synth.general(n, seed=77 + n)
    got = _to_string_order(_emulate(A, passes, n), n)
    want = oracle.coeffs_fwht(A)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_plans_exist_for_every_size(L, n):
    for dtype, prec in ((0, 0), (0, 1), (1, 0), (1, 2)):
        npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec))
        if 2 * n < _min_tile_bits(L):
            assert npass == 0
            continue
        passes = _parse(desc)
        assert 1 <= npass <= n and len(passes) == npass
        assert [p["b"] for p in passes] == list(np.cumsum([0] + [p["K"] for p in passes])[:-1])
        for p in passes:
            assert len(p["gbits"]) == p["D"] and p["ntiles"] == 2 ** (2 * n - p["D"])
            # lanes of every stage cover the three lowest tile bits, which are the
            # lowest column bits (128-byte runs of 16-byte elements)
            assert p["gbits"][:3] == [0, 1, 2]
    if n == 14:
        npass, _ = L.tpd_plan_describe(14, 0, L.options())
        assert npass == 3


def test_plan_choices_measured_on_gb300(L):
    """The planner's measured choices: complex128 n = 15 takes one 5-level pass
    over 2^13-element tiles between 2^12 and 2^11 ones, n = 16 four passes
    rather than two 2^13 passes; complex128 middle passes (int64 in and out)
    run on 2^11-element tiles, first and last passes on 2^12; the plain and
    fixed-point complex64 forms plan with 64-byte runs (n = 15 in three
    passes), the compensated one with 128-byte runs (four)."""
    def shape(n, dtype, prec):
        npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec))
        return [(p["K"], p["D"]) for p in _parse(desc)]
    assert shape(15, 0, 0) == [(6, 12), (5, 13), (4, 11)]
    assert shape(16, 0, 0) == [(4, 12), (4, 11), (4, 11), (4, 12)]
    assert shape(14, 0, 0) == [(6, 12), (4, 11), (4, 12)]
    assert shape(14, 1, 1) == [(6, 12), (4, 12), (4, 12)]       # complex64 keeps 2^12
    assert len(shape(15, 1, 3)) == 3 and len(shape(15, 1, 1)) == 3
    assert len(shape(15, 1, 2)) == 4


def test_pass_occupancy_choices(L):
    """CTAs per SM per pass: complex128 fixed point two (its passes convert
    both ways), a 2^13-element complex128 tile a two-CTA cluster (2), other 2^13
    tiles one CTA of 512 threads (1); compensated and fixed-point complex64
    three, except the fixed point's passes made only of two-level
    in-register stages on tiles below 2^12: two."""
    def ctas(n, dtype, prec):
        return [p["ctas"] for p in _parse(L.tpd_plan_describe(n, dtype, L.options(precision=prec))[1])]
    assert ctas(14, 0, 0) == [2, 2, 2]
    assert ctas(15, 0, 0) == [2, 2, 2]
    assert ctas(14, 0, 1) == [2, 2, 2]
    assert ctas(15, 1, 2) == [3, 3, 3, 3]
    assert ctas(15, 1, 3) == [3, 1, 2]
    assert ctas(14, 1, 3) == [3, 3, 3]
    assert ctas(14, 1, 2) == [3, 3, 3]
    assert ctas(14, 1, 1) == [2] * len(ctas(14, 1, 1))
    for n, dtype, prec in [(14, 1, 2), (15, 1, 2), (14, 1, 3), (15, 1, 3), (13, 1, 2)]:
        for p in _parse(L.tpd_plan_describe(n, dtype, L.options(precision=prec))[1]):
            pairs_only = len(p["stages"]) > 1 and all(s["npair"] == 2 and s["nshfl"] == 0 for s in p["stages"])
            two = pairs_only and prec == 3 and p["D"] < 12
            assert p["ctas"] == (1 if p["D"] > 12 else 2 if two else 3)


def test_tuned_defaults_apply_only_when_fields_are_zero(L):
    base = L.tpd_plan_describe(14, 0, L.options())
    small = L.tpd_plan_describe(14, 0, L.options(tile_bits=11))
    base13 = L.tpd_plan_describe(13, 0, L.options())
    base14_ieee = L.tpd_plan_describe(14, 0, L.options(precision=1))
    assert base != small
    try:
        assert L.tpd_tune_set(14, 0, 0, L.options(tile_bits=11)) == L.TPD_OK
        # a call that leaves the tuning fields at 0 (or passes no options) gets the tuned plan
        assert L.tpd_plan_describe(14, 0, L.options()) == small
        assert L.tpd_plan_describe(14, 0, None) == small
        # an explicit choice wins over the table; other keys are untouched
        assert L.tpd_plan_describe(14, 0, L.options(tile_bits=12)) == L.tpd_plan_describe(14, 0, L.options(
            tile_bits=12, max_levels=0))
        assert L.tpd_plan_describe(14, 0, L.options(max_levels=4))[1] != small[1]
        assert L.tpd_plan_describe(13, 0, L.options()) == base13
        assert L.tpd_plan_describe(14, 0, L.options(precision=1)) == base14_ieee
        # removing the entry restores the planner
        assert L.tpd_tune_set(14, 0, 0, None) == L.TPD_OK
        assert L.tpd_plan_describe(14, 0, L.options()) == base
        # bad keys and values are rejected
        assert L.tpd_tune_set(0, 0, 0, L.options()) == L.TPD_ERR_INVALID_ARG
        assert L.tpd_tune_set(14, 5, 0, L.options()) == L.TPD_ERR_INVALID_ARG
        assert L.tpd_tune_set(14, 0, 9, L.options()) == L.TPD_ERR_INVALID_ARG
        assert L.tpd_tune_set(14, 0, 0, L.options(tile_bits=5)) == L.TPD_ERR_INVALID_ARG
        assert L.tpd_tune_set(14, 0, 0, L.options(variant=9)) == L.TPD_ERR_INVALID_ARG
    finally:
        L.tpd_tune_clear()
    assert L.tpd_plan_describe(14, 0, L.options()) == base


def test_autotune_candidates_are_distinct_valid_plans(L):
    from paper_2310_13421_gb300 import autotune
    for n, dt, prec in ((14, "c128", 0), (8, "c128", 0), (15, "c64", 2), (4, "c64", 1)):
        cands = autotune.candidates(n, dt, prec)
        assert cands and cands[0] == dict(tile_bits=0, max_levels=0, variant=0, passes=cands[0]["passes"])
        keys = set()
        for c in cands:
            opt = L.options(precision=prec, tile_bits=c["tile_bits"], max_levels=c["max_levels"],
                            variant=c["variant"])
            npass, desc = L.tpd_plan_describe(n, autotune._DT[dt][0], opt)
            assert npass == c["passes"] >= 0
            keys.add((desc, c["variant"]))
        assert len(keys) == len(cands)


@pytest.mark.parametrize("n,dtype,prec", [(14, 0, 0), (15, 0, 0), (15, 1, 2), (13, 0, 0), (16, 1, 1)])
def test_l2_chunks_cover_each_fused_pass_once(L, n, dtype, prec):
    assert "l2 chunks" not in L.tpd_plan_describe(n, dtype, L.options(precision=prec))[1]   # off by default
    npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec, l2_chunk_mb=48))
    passes = _parse(desc)
    m = re.search(r"l2 chunks: passes=(\d+) fixed=([\d,]+)", desc)
    if m is None:
        assert n == 15 and dtype == 0 or n == 16                # no two passes fit 48 MB chunks
        return
    F = int(m.group(1))
    fixed = [int(x) for x in m.group(2).split(",")]
    assert 2 <= F < npass
    union = set()
    for p in passes[:F]:
        union |= set(p["gbits"])
    assert not union & set(fixed)                       # fixed bits lie outside every fused pass's tile
    elem = 16 if (dtype == 0 or prec >= 2) else 8
    assert 2 ** (2 * n - len(fixed)) * elem <= 48 << 20    # a chunk fits the default L2 budget
    # every tile of a fused pass lies in exactly one chunk: its tile-id bits hold all fixed bits
    for p in passes[:F]:
        rest = sorted(set(range(2 * n)) - set(p["gbits"]))
        assert set(fixed) <= set(rest)
    # off switch and the options that exclude chunking
    for opt in (L.options(precision=prec), L.options(precision=prec, skip_zero=True, l2_chunk_mb=48)):
        assert "l2 chunks" not in L.tpd_plan_describe(n, dtype, opt)[1]
