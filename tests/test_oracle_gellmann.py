"""CPU pins of the generalized Gell-Mann oracle (the qudit basis of Hermitian
symmetric, antisymmetric and diagonal matrices named in Sec. V as a candidate
for the method): Gell-Mann's eight 3x3 matrices and hand-derived coefficients
typed in tests/golden, dense Kronecker products, orthogonality, Parseval,
reconstruction, single elements, and the d = 2 case against the Pauli oracle."""
import os

import numpy as np
import pytest

import oracle
from oracle import core, kron
from paper_2310_13421_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rand(N, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))


def _value(tok):
    """a golden-file number: a complex literal, a fraction p/q, or isqrt3 = 1/sqrt(3) (optionally /q or -)"""
    sign = -1.0 if tok.startswith("-") else 1.0
    t = tok.lstrip("-")
    if t.startswith("isqrt3"):
        v = 1.0 / np.sqrt(3.0)
        if "/" in t:
            v /= float(t.split("/")[1])
        return sign * v
    if "/" in t:
        p, q = t.split("/")
        return sign * float(p) / float(q)
    return sign * complex(t)


def read_lambdas():
    out = []
    for line in open(os.path.join(GOLDEN, "gellmann_d3.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, *rows = line.split("|")
        name, r, c, factor = head.split()
        M = np.array([[complex(x) for x in row.split()] for row in rows], dtype=np.complex128)
        out.append((name, int(r), int(c), _value(factor) * M))
    return out


def test_d3_elements_are_gell_manns_lambdas():
    lam = read_lambdas()
    assert len(lam) == 8 and len({(r, c) for _, r, c, _ in lam}) == 8
    for name, r, c, M in lam:
        assert np.allclose(kron.gellmann_single(3, r, c), M, rtol=0, atol=1e-15), name   # sqrt(2/6) vs 1/sqrt(3): an ulp
    assert np.array_equal(kron.gellmann_single(3, 0, 0), np.eye(3))


def test_d3_unit_matrices_match_hand_derived_coefficients():
    for line in open(os.path.join(GOLDEN, "gellmann_d3_unit_matrices.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, *terms = line.split("|")
        a, b = (int(v) for v in head.split())
        E = np.zeros((3, 3), dtype=np.complex128)
        E[a, b] = 1.0
        want = np.zeros((3, 3), dtype=np.complex128)
        for t in terms:
            r, c, re, im = t.split()
            want[int(r), int(c)] = _value(re) + 1j * _value(im)
        got = core.gellmann_coeffs(E, 3)
        assert np.allclose(got, want, rtol=0, atol=2e-16), (a, b, got)


@pytest.mark.parametrize("d,n", [(2, 1), (2, 3), (3, 1), (3, 2), (4, 1), (4, 2), (5, 1)])
def test_gellmann_matches_kronecker(d, n):
    # random non-Hermitian input: a transposed or conjugated operand would fail
    A = rand(d ** n, 1600 + 10 * d + n)
    want = kron.gellmann_coeffs_kron(A, d)
    got = core.gellmann_coeffs(A, d)
    assert np.allclose(got, want, rtol=0, atol=1e-14)
    r = np.array([0, d ** n - 1, 1, d ** n // 2])
    c = np.array([0, d ** n - 1, d ** n - 1, 1])
    assert np.array_equal(core.gellmann_coeffs_at(A, d, r, c), got[r, c])


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_gellmann_kronecker_basis(d):
    # Hermitian, orthogonal with tr(G G') = N delta, traceless except the identity
    n = 2 if d < 5 else 1
    N = d ** n
    labels = [(r, c) for r in range(N) for c in range(N)]
    ops = [kron.gellmann_operator(d, kron._digits(r, d, n), kron._digits(c, d, n)) for r, c in labels]
    for G in ops:
        assert np.allclose(G, G.conj().T, atol=0)
    Gram = np.array([[np.trace(P @ Q) for Q in ops] for P in ops])
    assert np.allclose(Gram, np.diag(core.gellmann_norms(d, n).reshape(-1)), atol=1e-12)
    for (r, c), G in zip(labels, ops):
        if (r, c) != (0, 0) and n == 1:
            assert abs(np.trace(G)) <= 1e-15


@pytest.mark.parametrize("d,n", [(3, 3), (5, 2), (4, 3), (2, 5)])
def test_gellmann_parseval_and_reconstruction(d, n):
    A = rand(d ** n, 1700 + d + n)
    g = core.gellmann_coeffs(A, d)
    Nt = core.gellmann_norms(d, n)
    assert np.isclose(np.linalg.norm(A) ** 2, np.sum(Nt * np.abs(g) ** 2), rtol=1e-12)
    assert np.allclose(core.gellmann_compose(g, d), A, rtol=0, atol=1e-12)


@pytest.mark.parametrize("d,n", [(3, 2), (5, 1), (4, 2)])
def test_gellmann_single_element_is_a_unit_vector(d, n):
    N = d ** n
    g = np.random.default_rng(d + n)
    for r, c in [(0, 0), (N - 1, N - 1), (0, N - 1), (N - 1, 0), tuple(int(v) for v in g.integers(0, N, 2))]:
        G = kron.gellmann_operator(d, kron._digits(r, d, n), kron._digits(c, d, n))
        e = np.zeros((N, N), dtype=np.complex128)
        e[r, c] = 1.0
        assert np.allclose(core.gellmann_coeffs(G, d), e, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d,n", [(3, 3), (4, 2)])
def test_gellmann_hermitian_input_gives_real_coefficients(d, n):
    B = rand(d ** n, 1800 + d)
    A = (B + B.conj().T) / 2
    g = core.gellmann_coeffs(A, d)
    assert np.max(np.abs(g.imag)) <= 1e-14 * np.max(np.abs(g))
    assert np.max(np.abs(core.gellmann_coeffs(B, d).imag)) > 0.1      # and not for a general one


def pauli_rc_strings(n):
    """string index (base 4, t_1 most significant) of label (r, c): qubit
    n - b has symbol 2 r_b + c_b (I 0, X 1, Y 2, Z 3)"""
    N = 2 ** n
    r = np.repeat(np.arange(N), N)
    c = np.tile(np.arange(N), N)
    s = np.zeros(N * N, dtype=np.int64)
    for b in range(n):
        s += (2 * ((r >> b) & 1) + ((c >> b) & 1)) * 4 ** b
    return s


@pytest.mark.parametrize("n", [1, 3, 6])
def test_gellmann_d2_is_the_pauli_decomposition(n):
    # d = 2: I, X, Y, Z at (0,0), (0,1), (1,0), (1,1) with norm 2 each, so
    # g_(r,c) = 2^-n tr(sigma^t A) = w_t (Eq. 2); integers: bit-exact
    s = pauli_rc_strings(n)
    A = synth.general(n, seed=1900 + n)
    assert np.allclose(core.gellmann_coeffs(A, 2).reshape(-1), oracle.coeffs_fwht(A)[s], rtol=0, atol=1e-14)
    Ai = synth.int_general(n, seed=1910 + n)
    assert np.array_equal(core.gellmann_coeffs(Ai, 2).reshape(-1), oracle.coeffs_fwht(Ai)[s])


def _level_map(x, d):
    """One qudit level of the recursion on blocks x[..., r, c] (the d x d
    analogue of Eq. 4 for this basis), written from the single-qudit
    elements: y_(r,c) = tr(G_(r,c) x) / tr(G_(r,c)^2)."""
    y = np.empty_like(x)
    for r in range(d):
        for c in range(d):
            G = kron.gellmann_single(d, r, c)
            y[..., r, c] = np.einsum("uv,...vu->...", G, x) / np.trace(G @ G).real
    return y


@pytest.mark.parametrize("d,n", [(3, 3), (2, 4), (4, 2), (5, 2)])
def test_level_by_level_recursion_equals_the_trace_definition(d, n):
    # the reading behind the GPU path: the trace factorises over the qudits,
    # so applying the single-qudit map to every d x d block, one qudit at a
    # time (in any order), gives the coefficients of the trace definition,
    # each at the position of its label
    A = rand(d ** n, 2500 + d + n)
    want = core.gellmann_coeffs(A, d)
    for order in (range(n), reversed(range(n))):
        X = A.copy()
        for k in order:                       # digit k of row and column (stride d^k)
            s = d ** k
            h = d ** n // (d * s)
            B = X.reshape(h, d, s, h, d, s).transpose(0, 2, 3, 5, 1, 4)
            X = _level_map(B, d).transpose(0, 4, 1, 2, 5, 3).reshape(d ** n, d ** n)
        assert np.allclose(X, want, rtol=0, atol=1e-14)
