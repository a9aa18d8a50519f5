"""Per-coefficient accuracy on the GPU, against the oracle.

Every weight w_t with X-mask x is a signed sum of the 2^n entries A[r^x][r]
scaled by 2^-n (Eq. 2 through the one nonzero per row of a Pauli string).  Any
butterfly evaluation in IEEE arithmetic with unit roundoff u therefore obeys
the componentwise bound |err_t| <= gamma_n(u) m_x, with
m_x = 2^-n sum_r |A[r^x][r]| (each level forms sums of two terms, n levels;
Higham, Accuracy and Stability of Numerical Algorithms, Sec. 4.2): a weight's
error is set by the entries of its own X-mask only.

The block fixed point keeps that property.  A pass of K levels adds only
elements of one class (same X-mask on its levels, same passengers), and each
class sits on its own binary point, so every truncation is relative to
magnitudes of the weight's own X-mask.  complex128: the first pass truncates
an element by less than 2^(K-61) of its class's largest; a later pass puts a
class on its sources' largest binary point plus K, i.e. truncates by less than
2^(K_p-61) of the largest input of those sources in the pass before; the sums
are exact and each weight is rounded once, at the end.  Following a weight's
path through the passes gives |err_t| <= (sum_p 2^(2 K_p + K_{p-1} - 61) + u)
m_x with K_0 = 0 and u = 2^-53.  complex64: every pass rounds to float and
its classes take their own largest element: (sum_p 2^(2 K_p - 61) + P u) m_x,
u = 2^-24.  The oracle (Walsh-Hadamard form, fp64) adds its own
gamma_n(2^-53) m_x.  A shared per-tile binary point fails this on
diagonal-dominant matrices: the weak off-diagonal entries are truncated
relative to the strong diagonal of the same tile.

On top of the componentwise bound, every weight with |w_t| >= 1e-2 m_x is
checked to 1e-12 relative (complex128).
"""
import re

import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import U32, U64, assert_exact, rc_index_of_xz, to_string_order

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def levels_per_pass(n, dtype, prec):
    from paper_2310_13421_gb300 import _lib as L
    npass, desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec))
    if npass == 0:
        return [n]                     # whole matrix in one kernel: one class per X-mask
    return [int(e) - int(b) for b, e in re.findall(r"levels \[(\d+),(\d+)\)", desc)]


def m_of_x(A, xs):
    """m_x = 2^-n sum_r |A[r^x][r]| for each X-mask x."""
    N = A.shape[0]
    r = np.arange(N)
    return np.array([np.abs(A[r ^ int(x), r]).sum() / N for x in xs])


def m_per_string(A):
    """m_x of every string, string order (X-mask of string s from its base-4 digits)."""
    n = A.shape[0].bit_length() - 1
    s = np.arange(4 ** n, dtype=np.int64)
    x = np.zeros_like(s)
    for b in range(n):
        t = (s >> (2 * b)) & 3
        x |= ((t == 1) | (t == 2)).astype(np.int64) << b
    return m_of_x(A, np.arange(2 ** n))[x]


def bound(n, dtype, prec, u):
    Ks = levels_per_pass(n, dtype, prec)
    if dtype == 0:
        prev = [0] + Ks[:-1]
        fixed = sum(2.0 ** (2 * K + Kp - 61) for K, Kp in zip(Ks, prev)) + u
    else:
        fixed = sum(2.0 ** (2 * K - 61) for K in Ks) + len(Ks) * u
    return fixed + 1.01 * n * U64          # + the oracle's own gamma_n


def check(got, want, m, tol_m, what, rel=None):
    err = np.abs(got - want)
    lim = tol_m * m + 2.0 ** -1060
    bad = np.flatnonzero(err > lim)
    assert bad.size == 0, "%s: %d weights over the componentwise bound, worst %.3e of m_x (bound %.3e)" % (
        what, bad.size, np.max(err / np.maximum(m, 1e-300)), tol_m)
    if rel is not None:
        big = np.abs(want) >= 1e-2 * m
        assert big.sum() > 0.1 * big.size
        r = np.max(err[big] / np.abs(want[big]))
        assert r <= rel, "%s: per-coefficient relative error %.3e > %.1e" % (what, r, rel)


@pytest.mark.parametrize("scale", [1e5, 1e8])
def test_c128_fixed_diag_dominant_per_coefficient(tpd, scale):
    n = 10
    A = synth.diag_dominant(n, seed=5100, scale=scale)
    want = oracle.coeffs_fwht(A)
    m = m_per_string(A)
    for prec, code in (("fixed", 3), ("plain", 1)):
        got = to_string_order(host(tpd.decompose(gpu(A), precision=prec)), n)
        check(got, want, m, bound(n, 0, code, U64) if prec == "fixed" else 2.02 * n * U64,
              "n=10 diag %g %s" % (scale, prec), rel=1e-12)
        assert np.all(got.imag == 0), prec + ": Hermitian input, weights not exactly real"


def test_c128_fixed_diag_dominant_n14_sampled_rows(tpd):
    n = 14
    A = synth.diag_dominant(n, seed=5114, scale=1e8)
    W = host(tpd.decompose(gpu(A)))
    assert np.all(W.imag == 0)
    rng = np.random.default_rng(5)
    xs = np.concatenate([[0, 1, 2 ** (n - 1), 2 ** n - 1], rng.integers(1, 2 ** n, 12)]).astype(np.int64)
    want = oracle.coeffs_xrows(A, xs)
    z = np.arange(2 ** n)
    got = np.stack([W.reshape(-1)[rc_index_of_xz(x, z, n)] for x in xs])
    m = np.repeat(m_of_x(A, xs)[:, None], 2 ** n, axis=1)
    check(got.reshape(-1), want.reshape(-1), m.reshape(-1), bound(n, 0, 3, U64), "n=14 diag 1e8", rel=1e-12)


def test_c128_planted_string_far_below_diagonal(tpd):
    """A dominant diagonal plus 2^-40 X_j: the weight of X_j is exactly 2^-40
    (a dyadic sum inside its own X-mask), and every other weight off the
    diagonal's X-mask is exactly 0."""
    n = 12
    N = 2 ** n
    g = np.random.default_rng(7)
    A = np.zeros((N, N), dtype=np.complex128)
    A[np.diag_indices(N)] = np.round(g.standard_normal(N) * 2.0 ** 26)     # ~1e8, integers
    beta = 5                                        # qubit n - beta: X on row/column bit beta
    r = np.arange(N)
    A[r ^ (1 << beta), r] += 2.0 ** -40
    want = oracle.coeffs_fwht(A)
    s_x = int(oracle.string_of_xz(1 << beta, 0, n))
    assert want[s_x] == 2.0 ** -40
    for prec in ("fixed", "plain"):
        got = to_string_order(host(tpd.decompose(gpu(A), precision=prec)), n)
        assert_exact(got, want, prec)
        assert got[s_x] == 2.0 ** -40


def test_c128_dyadic_wide_range_one_tile(tpd):
    """1 and 2^-60 side by side in one tile, in different X-masks: every weight
    is a sum inside one X-mask of dyadic values and exact in fp64."""
    n = 8
    A = np.zeros((2 ** n, 2 ** n), dtype=np.complex128)
    A[0, 0] = 1.0
    A[0, 1] = 2.0 ** -60
    A[2, 0] = 3 * 2.0 ** -60
    A[1, 3] = -1j * 2.0 ** -61
    A[5, 5] = 0.5
    want = oracle.coeffs_fwht(A)
    for prec in ("fixed", "plain"):
        assert_exact(to_string_order(host(tpd.decompose(gpu(A), precision=prec)), n), want, prec)


def test_c64_diag_dominant_per_coefficient(tpd):
    """complex64 forms against the oracle on the same complex64 input: the
    fixed point within sum_p (2^(2K_p-61) + u32) m_x, compensated within
    (P+1) u32 m_x, plain fp32 within gamma_n(u32) m_x."""
    n = 10
    A = synth.diag_dominant(n, seed=5200, scale=1e5, dtype=np.complex64)
    want = oracle.coeffs_fwht(A.astype(np.complex128))
    m = m_per_string(A.astype(np.complex128))
    for prec, code in (("fixed", 3), ("compensated", 2), ("plain", 1)):
        got = to_string_order(host(tpd.decompose(gpu(A, torch.complex64), precision=prec)), n).astype(np.complex128)
        P = len(levels_per_pass(n, 1, code))
        tol = {"fixed": bound(n, 1, 3, U32), "compensated": (P + 1) * U32 * 1.01,
               "plain": n * U32 / (1 - n * U32)}[prec]
        check(got, want, m, tol, "c64 " + prec)


def test_sparse_coo_planted_string_far_below_diagonal(tpd):
    """The same planted case as COO input: one binary point per X-mask keeps
    the 2^-40 string exact beside a ~1e8 diagonal."""
    n = 12
    N = 2 ** n
    g = np.random.default_rng(8)
    d = np.round(g.standard_normal(N) * 2.0 ** 26)
    r = np.arange(N)
    beta = 3
    rows = np.concatenate([r, r ^ (1 << beta)]).astype(np.int32)
    cols = np.concatenate([r, r]).astype(np.int32)
    vals = np.concatenate([d, np.full(N, 2.0 ** -40)]).astype(np.complex128)
    A = np.zeros((N, N), dtype=np.complex128)
    A[rows, cols] += vals
    want = oracle.coeffs_fwht(A)
    keep = np.flatnonzero(want != 0)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    s, w = tpd.decompose_coo(t(rows, torch.int32), t(cols, torch.int32), t(vals, torch.complex128), n)
    assert host(s).tolist() == keep.tolist()
    assert_exact(host(w), want[keep])
    assert want[int(oracle.string_of_xz(1 << beta, 0, n))] == 2.0 ** -40
