"""CPU check of the thread-level index arithmetic of the pass kernels.

After a stage's shuffle levels the two lanes of a pair keep the row-1 output
they computed, so register e of lane L holds the element of lane L ^ Tw(e)'s
position (see shfl_level in tpd_pass.cuh).  The kernels fold that into the
per-register index weights of whatever follows the stage -- the shared-memory
exchange, the global store, the output class.  This test follows every
element through each stage of the library's plans (their stage maps read from
tpd_plan_describe) position by position, and checks that the weight formulas
the kernels use land each element exactly where its value belongs: every
shared-memory and global index of a tile is hit once, and each element's class
is the class of its position.  No GPU is involved.
"""
import re

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_2310_13421_gb300 import buildlib, _lib
    buildlib.build()
    _lib.load()
    return _lib


def parse(desc):
    passes = []
    for line in desc.strip().splitlines():
        if not line.startswith("pass "):
            continue
        head, *stages = line.split(" | ")
        m = re.match(r"pass \d+: levels \[(\d+),(\d+)\) D=(\d+) tiles=\d+ ctas=\d+ gbits=([\d,]+) cls=([\d,]+)", head)
        b, e, D, gbits, cls = m.groups()
        p = dict(D=int(D), K=int(e) - int(b), gbit=[int(x) for x in gbits.split(",")],
                 cls=[int(x) for x in cls.split(",")], stages=[])
        for st in stages:
            kv = dict(re.findall(r"(\w+)=([\d,]*)", st))
            ints = lambda k: [int(x) for x in kv[k].split(",")] if kv.get(k) else []
            p["stages"].append(dict(npair=int(kv["pairs"]), nshfl=int(kv["shfl"]), reg=ints("reg"),
                                    lane=ints("lane"), warp=ints("warp"), shfl_lane=ints("shfl_lane")))
        passes.append(p)
    return passes


def bits_of(x, n):
    return [(x >> i) & 1 for i in range(n)]


def lin(sel_bits, weights):
    """sum_i sel_bits[i] * weights[i] over numpy arrays of bits."""
    out = 0
    for b, w in zip(sel_bits, weights):
        out = out + b * w
    return out


def xlin(sel_bits, weights):
    out = 0
    for b, w in zip(sel_bits, weights):
        out = out ^ (b * w)
    return out


def check_stage(p, st):
    D = p["D"]
    nwarp = D - 9
    lane = np.arange(32)[:, None, None]
    warp = np.arange(1 << nwarp)[None, :, None]
    e = np.arange(16)[None, None, :]
    lb = bits_of(lane, 5)
    wb = bits_of(warp, nwarp)
    eb = bits_of(e, 4)
    one = lambda pos: 1 << pos
    # position of register e of each thread before the stage's levels
    pos = lin(lb, [one(x) for x in st["lane"]]) + lin(wb, [one(x) for x in st["warp"][:nwarp]]) + \
        lin(eb, [one(x) for x in st["reg"]])
    pos = np.broadcast_to(pos, (32, 1 << nwarp, 16)).copy()
    # the stage's shuffle levels, in order: a pair's row-1 register takes the
    # position its partner lane held
    for s in range(st["nshfl"]):
        rb = 2 * st["npair"] + s
        lbit = st["shfl_lane"][s]
        partner = pos[np.arange(32) ^ (1 << lbit)]
        row1 = ((np.arange(16) >> rb) & 1).astype(bool)
        pos[:, :, row1] = partner[:, :, row1]
    assert sorted(pos.reshape(-1).tolist()) == list(range(1 << D))

    def twisted(weights, lane_w, xor=False):
        w = [np.full((32, 1, 1), x, dtype=np.int64) for x in weights]
        for s in range(st["nshfl"]):
            rb = 2 * st["npair"] + s
            lbit = st["shfl_lane"][s]
            d = lane_w(st["lane"][lbit])
            if xor:
                w[rb] = w[rb] ^ d
            else:
                w[rb] = w[rb] + np.where(((np.arange(32) >> lbit) & 1)[:, None, None] == 1, -d, d)
        return w

    # shared-memory index (exchange source): thread_sidx + reg_off(twisted)
    t = lin(lb, [one(x) for x in st["lane"]]) + lin(wb, [one(x) for x in st["warp"][:nwarp]])
    idx = t + lin(eb, twisted([one(x) for x in st["reg"]], one))
    assert np.array_equal(np.broadcast_to(idx, pos.shape), pos)

    # global element index (store): thread_goff + reg_off(twisted), a linear map of the position
    g = lambda q: sum(((q >> b) & 1) << p["gbit"][b] for b in range(D))
    gw = lambda x: 1 << p["gbit"][x]
    gidx = lin(lb, [gw(x) for x in st["lane"]]) + lin(wb, [gw(x) for x in st["warp"][:nwarp]]) + \
        lin(eb, twisted([gw(x) for x in st["reg"]], gw))
    assert np.array_equal(np.broadcast_to(gidx, pos.shape), g(pos))

    # class (output rounding of the block fixed point): XOR-linear in the position
    cw = lambda x: p["cls"][x]
    cls_of = lambda q: np.bitwise_xor.reduce([((q >> b) & 1) * p["cls"][b] for b in range(D)])
    cidx = xlin(lb, [cw(x) for x in st["lane"]]) ^ xlin(wb, [cw(x) for x in st["warp"][:nwarp]]) ^ \
        xlin(eb, twisted([cw(x) for x in st["reg"]], cw, xor=True))
    assert np.array_equal(np.broadcast_to(cidx, pos.shape), cls_of(pos))


CASES = [(n, dtype, prec, tb, ml)
         for n in (5, 7, 9, 11, 12, 13, 14, 15, 16)
         for dtype, prec in ((0, 0), (1, 1), (1, 2), (1, 3))
         for tb, ml in ((0, 0), (11, 0), (13, 0), (0, 3), (0, 5))]


@pytest.mark.parametrize("n,dtype,prec,tb,ml", CASES)
def test_twisted_shuffle_indices(L, n, dtype, prec, tb, ml):
    npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec, tile_bits=tb, max_levels=ml))
    if npass <= 0:
        pytest.skip("whole-matrix kernel")
    passes = parse(desc)
    assert len(passes) == npass
    shuffled = 0
    for p in passes:
        for st in p["stages"]:
            check_stage(p, st)
            shuffled += st["nshfl"]
    if n >= 11 and tb == 0 and ml == 0:
        assert shuffled > 0        # the default plans' first passes shuffle
