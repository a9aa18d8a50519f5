"""GPU parity: libtpd.so (through the C ABI) against the CPU oracle.

Tolerances: complex128 1e-12 relative (each level is a scaled unitary map with
one rounding per output component, so fp64 stays within n u / (1 - n u) =
1.6e-15 at n = 14, and the fixed point rounds once), normwise and
elementwise against max|w|; integer and dyadic inputs bit-exact; complex64
against the oracle run on the same c64-rounded input, plain fp32 within
gamma_n = n u32 / (1 - n u32), compensated within (P+1) u32 for P passes.
"""
import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import U32, assert_close, assert_exact, rc_index_of_xz, rel_err, to_string_order

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL128 = 1e-12


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def gpu(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def npass(n, dtype=0, prec=0, **kw):
    from paper_2310_13421_gb300 import _lib as L
    return L.tpd_plan_describe(n, dtype, L.options(precision=prec, **kw))[0]


# ------------------------------------------------------------------ complex128

@pytest.mark.parametrize("precision", ["fixed", "plain"])
@pytest.mark.parametrize("n", list(range(1, 11)))
def test_c128_random_general(tpd, n, precision):
    A = synth.general(n, seed=2000 + n)
    got = to_string_order(host(tpd.decompose(gpu(A), precision=precision)), n)
    assert_close(got, oracle.coeffs_fwht(A), TOL128, "n=%d %s" % (n, precision))


@pytest.mark.parametrize("precision", ["fixed", "plain"])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9, 10, 11])
def test_c128_integer_bit_exact(tpd, n, precision):
    A = synth.int_general(n, seed=2100 + n)
    got = to_string_order(host(tpd.decompose(gpu(A), precision=precision)), n)
    assert_exact(got, oracle.coeffs_fwht(A), "n=%d %s" % (n, precision))


def test_n1_unit_matrices_golden(tpd):
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "n1_unit_matrices.txt"))
    for prec in ("fixed", "plain"):
        for row in rows:
            E = np.zeros((2, 2), dtype=np.complex128)
            E[int(row[0]), int(row[1])] = 1.0
            want = row[2::2] + 1j * row[3::2]
            assert_exact(to_string_order(host(tpd.decompose(gpu(E), precision=prec)), 1), want)


@pytest.mark.parametrize("precision", ["fixed", "plain"])
def test_c128_config_n12_integer_symmetric_bit_exact(tpd, precision):
    # real symmetric, entries uniform integers in [-8, 8], n = 12
    n = 12
    A = synth.int_symmetric(n, seed=3003)
    got = to_string_order(host(tpd.decompose(gpu(A), precision=precision)), n)
    want = oracle.coeffs_fwht(A)
    assert_exact(got, want, "n=12 int symmetric")
    # odd number of Y factors: exactly zero (footnote of Sec. II.B)
    s = np.arange(4 ** n)
    ny = np.zeros_like(s)
    for b in range(n):
        ny += ((s >> (2 * b)) & 3) == 2
    assert np.all(got[ny % 2 == 1] == 0)


@pytest.mark.parametrize("precision", ["fixed", "plain"])
def test_c128_n12_hermitian_full(tpd, precision):
    n = 12
    A = synth.hermitian(n, seed=3012)
    got = to_string_order(host(tpd.decompose(gpu(A), precision=precision)), n)
    assert_close(got, oracle.coeffs_fwht(A), TOL128, "n=12")
    # Hermitian: exactly real in both arithmetics (IEEE adds, and the fixed
    # point's truncation toward zero and round to nearest, are odd functions,
    # and conjugate partners share their class's binary point)
    assert np.all(got.imag == 0)


def test_c128_config_n6(tpd):
    # 64x64 Hermitian, N(0,1) parts: all 4096 weights
    n = 6
    A = synth.hermitian(n, seed=1001)
    for prec in ("fixed", "plain"):
        got = to_string_order(host(tpd.decompose(gpu(A), precision=prec)), n)
        assert_close(got, oracle.coeffs(A), TOL128, "n=6 " + prec)


@pytest.mark.parametrize("opt", [dict(tile_bits=9), dict(tile_bits=10), dict(tile_bits=11), dict(tile_bits=13),
                                 dict(max_levels=1), dict(max_levels=2), dict(max_levels=3),
                                 dict(max_levels=5), dict(tile_bits=12, max_levels=4), dict(variant=1),
                                 dict(variant=2), dict(tile_bits=11, variant=2)])
def test_c128_plan_variants(tpd, opt):
    n = 10
    A = synth.general(n, seed=4000)
    want = oracle.coeffs_fwht(A)
    for prec in ("fixed", "plain"):
        got = to_string_order(host(tpd.decompose(gpu(A), precision=prec, **opt)), n)
        assert_close(got, want, TOL128, str(opt))
    Ai = synth.int_general(n, seed=4001)
    assert_exact(to_string_order(host(tpd.decompose(gpu(Ai), **opt)), n), oracle.coeffs_fwht(Ai))


def test_c128_magnitude_extremes(tpd):
    # tiny (subnormal-range products) and huge entries go through the fixed
    # point's exponent handling; compare with the oracle on the same input
    n = 8
    base = synth.general(n, seed=4100)
    for scale in (1e-300, 1e-310, 1e300, 2.0 ** -1070):
        A = base * scale
        want = oracle.coeffs_fwht(A)
        got = to_string_order(host(tpd.decompose(gpu(A), precision="fixed")), n)
        if scale < 1e-305:
            # results sit in the subnormal range: absolute error half an ulp of the smallest normal
            assert np.max(np.abs(got - want)) <= 2.0 ** -1074 * 2 ** n
        else:
            # compare rescaled copies (norms of 1e300-sized vectors overflow)
            assert_close(got / scale, want / scale, TOL128, "scale %g" % scale)
    # wide dynamic range inside one tile
    A = base.copy()
    A[::3, ::5] *= 1e12
    assert_close(to_string_order(host(tpd.decompose(gpu(A))), n), oracle.coeffs_fwht(A), TOL128, "mixed")


@pytest.mark.parametrize("n,opt", [(8, {}), (12, dict(tile_bits=13))])   # 12: two-CTA cluster tiles
def test_c128_nonfinite_tiles_follow_ieee(tpd, n, opt):
    A = synth.general(n, seed=4200)
    A[3, 7] = np.inf
    A[100, 5] = np.nan
    fixed = host(tpd.decompose(gpu(A), precision="fixed", **opt))
    plain = host(tpd.decompose(gpu(A), precision="plain", **opt))
    assert np.array_equal(np.isnan(fixed), np.isnan(plain))
    assert np.array_equal(np.isinf(fixed), np.isinf(plain))
    fin = np.isfinite(fixed) & np.isfinite(plain)
    assert fin.any() and np.allclose(fixed[fin], plain[fin], rtol=1e-12, atol=1e-12)
    if opt:
        # the Inf/NaN fallback of a cluster tile: the same bits as one 512-thread CTA (NaN payloads aside)
        one = host(tpd.decompose(gpu(A), precision="fixed", variant=1, **opt))
        assert np.array_equal(np.isnan(fixed), np.isnan(one))
        ok = ~np.isnan(fixed)
        assert np.array_equal(fixed[ok], one[ok])


@pytest.mark.parametrize("n,opt", [(11, {}), (12, dict(tile_bits=13)), (13, dict(tile_bits=13, max_levels=5))])
def test_c128_cluster_tiles_match_one_cta(tpd, n, opt):
    """Complex128 tiles of 2^13 elements run as a cluster of two 256-thread
    CTAs; one 512-thread CTA per tile (variant 1) computes the same sums in
    the same order: identical bits, decomposition and composition, with and
    without zero skipping (also on a matrix with all-zero tiles), fixed
    point and fp64; and the oracle where it is cheap."""
    from paper_2310_13421_gb300 import _lib as L
    assert "D=13" in L.tpd_plan_describe(n, 0, L.options(**opt))[1]
    A = synth.general(n, seed=4100 + n)
    H = synth.heisenberg(n, *synth.heisenberg_params(n, seed=4150 + n))
    for prec in ("fixed", "plain"):
        for M in (A, H):
            for skip in (False, True):
                cl = host(tpd.decompose(gpu(M), precision=prec, skip_zero=skip, **opt))
                one = host(tpd.decompose(gpu(M), precision=prec, skip_zero=skip, variant=1, **opt))
                assert_exact(cl, one, "decompose n=%d %s skip=%s" % (n, prec, skip))
        c_cl = host(tpd.compose(gpu(A), precision=prec, **opt))
        c_one = host(tpd.compose(gpu(A), precision=prec, variant=1, **opt))
        assert_exact(c_cl, c_one, "compose n=%d %s" % (n, prec))
        if n <= 12:
            got = to_string_order(host(tpd.decompose(gpu(A), precision=prec, **opt)), n)
            assert_close(got, oracle.coeffs_fwht(A), TOL128, "oracle n=%d %s" % (n, prec))


def test_c128_zero_matrix_and_skip(tpd):
    for n in (3, 7, 10):
        Z = torch.zeros((2 ** n, 2 ** n), dtype=torch.complex128, device="cuda")
        for skip in (False, True):
            out = tpd.decompose(Z, skip_zero=skip)
            assert torch.count_nonzero(out).item() == 0


@pytest.mark.parametrize("n", [6, 9, 10])
def test_skip_zero_identical_results(tpd, n):
    for A in (synth.general(n, seed=4300 + n), synth.heisenberg(n, *synth.heisenberg_params(n, seed=n))):
        a = host(tpd.decompose(gpu(A), skip_zero=False))
        b = host(tpd.decompose(gpu(A), skip_zero=True))
        assert_exact(b, a)


@pytest.mark.parametrize("n", [5, 8, 10, 12])
def test_planted_heisenberg_exact(tpd, n):
    J, h = synth.heisenberg_params(n, seed=5000 + n)
    H = synth.heisenberg(n, J, h)
    terms = synth.heisenberg_terms(n, J, h)
    for prec in ("fixed", "plain"):
        got = to_string_order(host(tpd.decompose(gpu(H), precision=prec, skip_zero=True)), n)
        want = np.zeros(4 ** n, dtype=np.complex128)
        for t, v in terms.items():
            want[synth.string_index(t)] = v
        assert_exact(got, want, "heisenberg n=%d" % n)


def test_tfim_eq7_first_level_and_terms(tpd):
    # Eq. 8: after the first qubit level (the top one), the CMWs are H_{n-1}, -J g I,
    # 0 and -J Z; the full decomposition has the 2n-1 terms of Eq. 7
    n, J, g = 8, 0.75, -1.25
    H = synth.tfim(n, J, g)
    got = to_string_order(host(tpd.decompose(gpu(H), skip_zero=True)), n)
    want = np.zeros(4 ** n, dtype=np.complex128)
    for t, v in synth.tfim_terms(n, J, g).items():
        want[synth.string_index(t)] = v
    assert_exact(got, want)


# ------------------------------------------------------------------ complex64

@pytest.mark.parametrize("n", [3, 5, 8, 10, 11])
def test_c64_plain_and_compensated(tpd, n):
    A64 = synth.hermitian(n, seed=6000 + n, dtype=np.complex64)
    want = oracle.coeffs_fwht(A64.astype(np.complex128))
    plain = to_string_order(host(tpd.decompose(gpu(A64, torch.complex64), precision="plain")), n)
    comp = to_string_order(host(tpd.decompose(gpu(A64, torch.complex64), precision="compensated")), n)
    P = max(npass(n, 1, 2), 1)
    g_plain = n * U32 / (1 - n * U32)
    g_comp = (P + 1) * U32 / (1 - (P + 1) * U32)
    e_plain, e_comp = rel_err(plain, want), rel_err(comp, want)
    assert e_plain <= g_plain, e_plain
    assert e_comp <= g_comp, e_comp
    if n >= 8:
        assert e_comp < e_plain
    # complex64 block fixed point: each pass sums exactly and rounds once, so
    # every pass adds at most u32 relative error (normwise): <= P u32 in all
    fixed = to_string_order(host(tpd.decompose(gpu(A64, torch.complex64), precision="fixed")), n)
    Pf = max(npass(n, 1, 3), 1)
    e_fixed = rel_err(fixed, want)
    assert e_fixed <= Pf * U32 / (1 - Pf * U32), e_fixed


@pytest.mark.parametrize("n", [4, 9, 10])
def test_c64_integer_bit_exact(tpd, n):
    A = synth.int_general(n, seed=6100 + n)
    want = oracle.coeffs_fwht(A)
    for prec in ("plain", "compensated", "fixed"):
        got = to_string_order(host(tpd.decompose(gpu(A, torch.complex64), precision=prec)), n)
        assert_exact(got.astype(np.complex128), want, prec)


# ------------------------------------------------------------------ composition

@pytest.mark.parametrize("precision", ["fixed", "plain"])
@pytest.mark.parametrize("n", [1, 3, 6, 9, 10])
def test_compose_matches_oracle(tpd, n, precision):
    W = synth.general(n, seed=7000 + n)  # weights in RC layout
    want = oracle.compose_fwht(to_string_order(W, n), n)
    got = host(tpd.compose(gpu(W), precision=precision))
    assert_close(got, want, TOL128, "compose n=%d" % n)
    adj = host(tpd.compose(gpu(W), scale=2.0 ** -n, precision=precision))
    assert_close(adj, want * 2.0 ** -n, TOL128, "adjoint n=%d" % n)


@pytest.mark.parametrize("n", [2, 7, 10, 12])
def test_roundtrip_exact_on_integers(tpd, n):
    A = synth.int_general(n, seed=7100 + n)
    c = tpd.decompose(gpu(A))
    assert_exact(host(tpd.compose(c)), A)
    c64 = tpd.decompose(gpu(A, torch.complex64), precision="compensated")
    assert_exact(host(tpd.compose(c64, precision="compensated")).astype(np.complex128), A)


def test_compose_non_power_of_two_scale(tpd):
    n = 9
    W = synth.general(n, seed=7200)
    want = 0.3 * oracle.compose_fwht(to_string_order(W, n), n)
    for prec in ("fixed", "plain"):
        assert_close(host(tpd.compose(gpu(W), scale=0.3, precision=prec)), want, TOL128)


def test_adjoint_dot_product(tpd):
    n = 10
    A = gpu(synth.general(n, seed=7300))
    G = gpu(synth.general(n, seed=7301))
    lhs = torch.vdot(tpd.decompose(A).reshape(-1), G.reshape(-1)).item()
    rhs = torch.vdot(A.reshape(-1), tpd.compose(G, scale=2.0 ** -n).reshape(-1)).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ------------------------------------------------------------------ batched

def test_batched_mixed_sizes(tpd):
    rng = np.random.default_rng(8000)
    # n = 11: a second pass of 2^13-element tiles (two-CTA clusters); n = 12: the largest batched size
    ns = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 11] + list(rng.integers(1, 11, size=22))
    mats = [synth.general(int(n), seed=8000 + i) for i, n in enumerate(ns)]
    for prec in ("fixed", "plain"):
        outs = tpd.decompose_batched([gpu(m) for m in mats], precision=prec)
        for m, o, n in zip(mats, outs, ns):
            assert_close(to_string_order(host(o), int(n)), oracle.coeffs_fwht(m), TOL128, "batched n=%d" % n)
    ints = [synth.int_general(int(n), seed=8100 + i) for i, n in enumerate(ns)]
    outs = tpd.decompose_batched([gpu(m) for m in ints])
    for m, o, n in zip(ints, outs, ns):
        assert_exact(to_string_order(host(o), int(n)), oracle.coeffs_fwht(m))
    # batched composition with the adjoint scaling inverts up to 2^-n: C(D(A)) = A
    back = tpd.compose_batched(outs)
    for m, b in zip(ints, back):
        assert_exact(host(b), m)


def test_batched_c64(tpd):
    ns = [3, 5, 8, 10, 4, 9]
    mats = [synth.hermitian(n, seed=8200 + n, dtype=np.complex64) for n in ns]
    outs = tpd.decompose_batched([gpu(m, torch.complex64) for m in mats], precision="compensated")
    for m, o, n in zip(mats, outs, ns):
        P = max(npass(n, 1, 2), 1)
        assert rel_err(to_string_order(host(o), n), oracle.coeffs_fwht(m.astype(np.complex128))) <= (P + 1) * U32 * 1.01


def test_batched_cuda_graph_replay(tpd):
    ns = [3, 6, 8, 10]
    mats = [synth.general(n, seed=8300 + n) for n in ns]
    work = [gpu(m) for m in mats]
    pristine = [w.clone() for w in work]
    batch = tpd.Batch(work)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.decompose(stream=s)   # warm-up (plans, attributes) outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.decompose()
    for rep in range(3):
        for w, p in zip(work, pristine):
            w.copy_(p)
        g.replay()
        torch.cuda.synchronize()
        for m, w, n in zip(mats, work, ns):
            assert_close(to_string_order(host(w), n), oracle.coeffs_fwht(m), TOL128, "graph n=%d" % n)


# ------------------------------------------------------------------ autograd

def test_autograd_matches_oracle_gradient(tpd):
    n = 8
    A = synth.hermitian(n, seed=9000)
    w = synth.loss_weights(n, seed=9001)
    wt_rc = np.empty(4 ** n)
    from _helpers import rc_positions
    wt_rc[rc_positions(n)] = w
    At = gpu(A).requires_grad_(True)
    c = tpd.tpd(At)
    loss = (torch.from_numpy(wt_rc).cuda().reshape(c.shape) * c.abs() ** 2).sum()
    loss.backward()
    assert_close(host(At.grad), oracle.grad_weighted_sq(A, w), TOL128, "grad")


# ------------------------------------------------------------------ autotuner

def test_autotune_registers_a_plan_that_matches_oracle(tpd, tmp_path):
    from paper_2310_13421_gb300 import autotune, _lib as L
    cache = str(tmp_path / "tune.json")
    try:
        res = autotune.tune(9, "c128", "default", reps=2, batch_bytes=8 << 20, cache=cache)
        assert res["best"] and res["ms"] > 0 and len(res["tried"]) >= 2
        res64 = autotune.tune(11, "c64", "compensated", reps=2, cache=cache)
        L.tpd_tune_clear()
        assert autotune.load(cache) == 2
        # calls that leave the tuning fields at 0 now run the tuned plans
        A = synth.general(9, seed=9100)
        out = tpd.decompose(gpu(A))
        assert_close(to_string_order(host(out), 9), oracle.coeffs_fwht(A), TOL128, "tuned n=9")
        ns = [9, 9, 9]
        mats = [synth.int_general(9, seed=9110 + i) for i in range(3)]
        outs = tpd.decompose_batched([gpu(m) for m in mats])
        for m, o in zip(mats, outs):
            assert_exact(to_string_order(host(o), 9), oracle.coeffs_fwht(m))
        B = synth.hermitian(11, seed=9120, dtype=np.complex64)
        o = tpd.decompose(gpu(B, torch.complex64), precision="compensated")
        P = max(npass(11, 1, 2, **res64["best"]), 1)
        assert rel_err(to_string_order(host(o), 11), oracle.coeffs_fwht(B.astype(np.complex128))) <= \
            (P + 1) * U32 * 1.01
    finally:
        L.tpd_tune_clear()


# ------------------------------------------------------------------ layout and norms

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 10])
def test_string_layout_is_the_base4_order(tpd, n):
    from _helpers import rc_positions
    for dt, npdt in ((torch.complex128, np.complex128), (torch.complex64, np.complex64)):
        A = synth.general(n, seed=9300 + n).astype(npdt)
        W = tpd.decompose(gpu(A, dt))
        S = tpd.to_string_layout(W)
        w = host(W).reshape(-1)
        assert_exact(host(S), w[rc_positions(n)], "string layout n=%d" % n)
        assert_exact(host(tpd.from_string_layout(S)), host(W), "back to RC n=%d" % n)
        if dt == torch.complex128:
            assert_close(host(S), oracle.coeffs_fwht(A), TOL128, "string order vs oracle n=%d" % n)


def test_sum_squares_parseval_and_determinism(tpd):
    for n in (3, 9, 12):
        A = synth.general(n, seed=9400 + n)
        At = gpu(A)
        W = tpd.decompose(At)
        a2 = tpd.sum_squares(At)
        w2 = tpd.sum_squares(W)
        a2_host = float(np.sum(np.abs(A) ** 2))
        assert abs(float(a2) - a2_host) <= 1e-13 * a2_host
        # Parseval: ||A||_F^2 = 2^n sum |w|^2
        assert abs(float(w2) * 2 ** n - a2_host) <= 1e-12 * a2_host
        assert float(tpd.sum_squares(At)) == float(a2)          # same bits every call
    B = synth.hermitian(10, seed=9410, dtype=np.complex64)
    b2 = float(tpd.sum_squares(gpu(B, torch.complex64)))
    want = float(np.sum(np.abs(B.astype(np.complex128)) ** 2))
    assert abs(b2 - want) <= 1e-12 * want
    empty = torch.empty(0, dtype=torch.complex128, device="cuda")
    assert float(tpd.sum_squares(empty)) == 0.0


@pytest.mark.parametrize("n", [5, 9, 11])
def test_c64_fixed_rounding_and_extremes(tpd, n):
    A = synth.general(n, seed=6200 + n).astype(np.complex64)
    got = to_string_order(host(tpd.decompose(gpu(A, torch.complex64), precision="fixed")), n)
    want = oracle.coeffs_fwht(A.astype(np.complex128))
    if npass(n, 1, 3) == 1:
        # one pass: the exact sum, rounded once to the nearest float -- within the
        # unit roundoff u32 = 2^-24 relative to the exact weight in each component
        # (plus the truncation of components far below the tile's largest, < 2^-30 of it)
        tiny = 2.0 ** -30 * np.max(np.abs(want))
        for part in (np.real, np.imag):
            assert np.all(np.abs(part(got) - part(want)) <= U32 * np.abs(part(want)) + tiny)
    # magnitudes near the ends of the float range
    for scale in (2.0 ** 100, 2.0 ** -100):
        B = A * np.float32(scale)
        g2 = to_string_order(host(tpd.decompose(gpu(B, torch.complex64), precision="fixed")), n)
        w2 = oracle.coeffs_fwht(B.astype(np.complex128))
        assert rel_err(g2, w2) <= max(npass(n, 1, 3), 1) * U32 * 1.01
    # composition of the weights gives A back within the rounding of both directions
    C = tpd.compose(tpd.decompose(gpu(A, torch.complex64), precision="fixed"), precision="fixed")
    assert rel_err(host(C), A) <= 2 * max(npass(n, 1, 3), 1) * U32 * 1.01


def test_nonzero_list_is_the_papers_list(tpd):
    # planted Hamiltonians: exactly the planted strings, in string order, exact weights
    for n in (2, 5, 10):
        J, h = synth.heisenberg_params(n, seed=9500 + n)
        terms = synth.heisenberg_terms(n, J, h)
        want = sorted((synth.string_index(t), v) for t, v in terms.items())
        s, w = tpd.nonzero_list(tpd.decompose(gpu(synth.heisenberg(n, J, h))))
        assert host(s).tolist() == [k for k, _ in want]
        assert_exact(host(w), np.array([v for _, v in want], dtype=np.complex128))
    # a threshold, complex64, and a capacity smaller than the list
    n = 6
    A = synth.general(n, seed=9510).astype(np.complex64)
    W = tpd.decompose(gpu(A, torch.complex64))
    full = to_string_order(host(W), n)
    tol = 0.05
    keep = np.flatnonzero((np.abs(full.real) > tol) | (np.abs(full.imag) > tol))
    s, w = tpd.nonzero_list(W, tol=tol)
    assert host(s).tolist() == keep.tolist()
    assert_exact(host(w), full[keep])
    s2, w2, cnt = tpd.nonzero_list(W, tol=tol, capacity=10)
    assert int(host(cnt)[0]) == keep.size
    assert host(s2).tolist() == keep[:10].tolist()


@pytest.mark.parametrize("n,mb", [(12, 1), (12, 8), (13, 4)])
def test_l2_chunked_passes_identical(tpd, n, mb):
    # the first passes run chunk by chunk: every tile is computed exactly as in
    # the plain launch sequence, so the weights are the same bits
    A = synth.general(n, seed=9800 + n)
    for prec in ("fixed", "plain"):
        plain = host(tpd.decompose(gpu(A), precision=prec))
        chunked = host(tpd.decompose(gpu(A), precision=prec, l2_chunk_mb=mb))
        assert_exact(chunked, plain, "chunked n=%d %s" % (n, prec))
    assert_close(to_string_order(chunked, n), oracle.coeffs_fwht(A), TOL128, "vs oracle")


@pytest.mark.parametrize("n,pinned,inplace", [(6, True, False), (10, True, True), (11, False, False)])
def test_decompose_from_host_buffers(tpd, n, pinned, inplace):
    # tpd_decompose_host: host -> device copy, decomposition and device -> host
    # copy, all enqueued on the stream (the end-to-end path of the benchmark)
    from paper_2310_13421_gb300 import _lib as L
    A = synth.general(n, seed=9900 + n)
    src = torch.from_numpy(A.copy())
    if pinned:
        src = src.pin_memory()
    dst = src if inplace else torch.empty_like(src)
    dev = torch.empty(A.shape, dtype=torch.complex128, device="cuda")
    wsb = L.tpd_workspace_size(n, L.TPD_C128, None)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    st = L.tpd_decompose_host(src.data_ptr(), dst.data_ptr(), dev.data_ptr(), n, L.TPD_C128, None, ws.data_ptr(), wsb,
                              s.cuda_stream)
    assert st == L.TPD_OK
    torch.cuda.synchronize()
    got = dst.numpy()
    assert_exact(got, host(dev))                       # the host copy is the device result
    assert_close(to_string_order(got, n), oracle.coeffs_fwht(A), TOL128, "host path n=%d" % n)


def test_single_decomposition_in_cuda_graph(tpd):
    # the whole launch sequence of one call is captured and replayed
    n = 12
    A = synth.general(n, seed=9950)
    src = gpu(A)
    work = src.clone()
    from paper_2310_13421_gb300 import _lib as L
    for prec, skip in (("fixed", False), ("plain", True)):
        opt = tpd.make_options(prec, skip)
        wsb = L.tpd_workspace_size(n, L.TPD_C128, opt)
        ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            st = L.tpd_decompose(work.data_ptr(), n, L.TPD_C128, opt, ws.data_ptr(), wsb, s.cuda_stream)
            assert st == L.TPD_OK
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            st = L.tpd_decompose(work.data_ptr(), n, L.TPD_C128, opt, ws.data_ptr(), wsb,
                                 torch.cuda.current_stream().cuda_stream)
        assert st == L.TPD_OK
        for _ in range(2):
            work.copy_(src)
            g.replay()
            assert_close(to_string_order(host(work), n), oracle.coeffs_fwht(A), TOL128, "graph %s" % prec)
