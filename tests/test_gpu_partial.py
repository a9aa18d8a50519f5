"""GPU: partial decomposition (Alg. 3) -- only the weights of a list of
strings -- against the CPU oracle evaluated at those strings, bit-identical to
the full decomposition, on planted Hamiltonians, and in a CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import U32, assert_close, assert_exact, rc_positions, rel_err

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


def request(n, count, seed):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, 4 ** n, size=count, dtype=np.int64)
    s[:3] = [0, 4 ** n - 1, s[3]]          # the all-I and all-Z strings, and a duplicate
    return [int(x) for x in s]


@pytest.mark.parametrize("n", [2, 5, 8, 10, 11, 12])    # n = 11: a pass of 2^13-element cluster tiles
@pytest.mark.parametrize("precision", ["fixed", "plain"])
def test_partial_matches_oracle_and_full(tpd, n, precision):
    A = synth.general(n, seed=9600 + n)
    strings = request(n, 64, 9610 + n)
    part = tpd.Partial(n, strings, precision=precision)
    got = host(part.decompose(gpu(A)))
    full = host(tpd.decompose(gpu(A), precision=precision)).reshape(-1)
    # the same sums in the same order as the full decomposition; in the fixed
    # point every class a requested weight depends on lies inside its
    # dependency cone, so it has the same binary point as in the full run
    assert_exact(got, full[rc_positions(n)[strings]], "partial vs full n=%d" % n)
    assert_close(got, oracle.coeffs_at(A, strings), TOL128, "partial vs oracle n=%d" % n)
    Ai = synth.int_general(n, seed=9620 + n)       # integer input: exact either way
    got_i = host(part.decompose(gpu(Ai)))
    assert_exact(got_i, host(tpd.decompose(gpu(Ai), precision=precision)).reshape(-1)[rc_positions(n)[strings]])


@pytest.mark.parametrize("precision", ["plain", "compensated"])
def test_partial_c64(tpd, precision):
    n = 11
    A = synth.hermitian(n, seed=9620, dtype=np.complex64)
    strings = request(n, 200, 9621)
    got = host(tpd.Partial(n, strings, dtype=torch.complex64, precision=precision).decompose(gpu(A, torch.complex64)))
    full = host(tpd.decompose(gpu(A, torch.complex64), precision=precision)).reshape(-1)
    assert_exact(got, full[rc_positions(n)[strings]])
    want = oracle.coeffs_at(A.astype(np.complex128), strings)
    assert np.max(np.abs(got - want)) <= 8 * n * U32 * np.max(np.abs(oracle.coeffs_fwht(A.astype(np.complex128))))


def test_partial_planted_heisenberg(tpd):
    n = 12
    J, h = synth.heisenberg_params(n, seed=9630)
    H = synth.heisenberg(n, J, h)
    terms = synth.heisenberg_terms(n, J, h)
    # planted strings + three zero weights: I..I (traceless H), X on qubit 1 alone, Z..ZY
    strings = [synth.string_index(t) for t in terms] + [0, 4 ** (n - 1), 4 ** n - 2]
    want = np.array([terms[t] for t in terms] + [0.0, 0.0, 0.0], dtype=np.complex128)
    got = host(tpd.Partial(n, strings).decompose(gpu(H)))
    assert_exact(got, want, "planted")


def test_partial_skips_tiles(tpd):
    # a dense input and a narrow request: a position inside no needed tile of
    # any pass is never written, so it still holds the input's bits, while the
    # requested weights are the full decomposition's
    n = 12
    A = synth.general(n, seed=9635)
    strings = request(n, 8, 9636)
    Ad = gpu(A)
    got = host(tpd.Partial(n, strings).decompose(Ad, inplace=True))
    full = host(tpd.decompose(gpu(A))).reshape(-1)
    assert_exact(got, full[rc_positions(n)[strings]])
    untouched = np.mean(host(Ad).reshape(-1).view(np.int64) == A.reshape(-1).view(np.int64))
    assert untouched > 0.5, "only %.3f of the positions kept their input bits" % untouched


def test_partial_graph_replay(tpd):
    n = 10
    A = synth.general(n, seed=9640)
    strings = request(n, 32, 9641)
    part = tpd.Partial(n, strings)
    src = gpu(A)
    work = src.clone()
    out = torch.empty(len(strings), dtype=torch.complex128, device="cuda")
    part.decompose(work, inplace=True, out=out)          # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        part.decompose(work, inplace=True, out=out)
    want = oracle.coeffs_at(A, strings)
    for _ in range(2):
        work.copy_(src)
        out.zero_()
        g.replay()
        assert_close(host(out), want, TOL128, "graph")
