"""CPU pins of the Weyl-basis oracle (the qudit basis of clock and shift
operators named in Sec. V as the next candidate for the method): dense
Kronecker products, orthogonality, Parseval, reconstruction, single operators,
the d = 2 case against the Pauli oracle, and the conjugation symmetry of
Hermitian inputs."""
import numpy as np
import pytest

import oracle
from oracle import core, kron
from paper_2310_13421_gb300 import synth


def rand(N, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))


def neg(x, d, n):
    """digit-wise -x mod d"""
    out, p = 0, 1
    for _ in range(n):
        out += ((-(x % d)) % d) * p
        x //= d
        p *= d
    return out


def dot(x, y, d, n):
    s = 0
    for _ in range(n):
        s += (x % d) * (y % d)
        x //= d
        y //= d
    return s % d


@pytest.mark.parametrize("d,n", [(3, 1), (3, 2), (2, 1), (2, 3), (4, 1), (4, 2), (5, 1)])
def test_weyl_matches_kronecker(d, n):
    # random non-Hermitian input: a transposed or conjugated operand would fail
    A = rand(d ** n, 600 + 10 * d + n)
    want = kron.weyl_coeffs_kron(A, d)
    assert np.allclose(core.weyl_coeffs(A, d), want, rtol=0, atol=1e-14)
    assert np.allclose(core.weyl_coeffs_dft(A, d), want, rtol=0, atol=1e-14)


@pytest.mark.parametrize("d", [2, 3, 5])
def test_weyl_kronecker_basis_is_orthogonal(d):
    n = 2 if d < 5 else 1
    N = d ** n
    ops = [kron.weyl_operator(d, kron._digits(a, d, n), kron._digits(b, d, n)) for a in range(N) for b in range(N)]
    G = np.array([[np.trace(P.conj().T @ Q) for Q in ops] for P in ops])
    assert np.allclose(G, N * np.eye(N * N), atol=1e-12)


@pytest.mark.parametrize("d,n", [(3, 3), (3, 5), (5, 2), (2, 6)])
def test_weyl_parseval_and_reconstruction(d, n):
    A = rand(d ** n, 700 + d + n)
    c = core.weyl_coeffs_dft(A, d)
    assert np.isclose(np.linalg.norm(A) ** 2, d ** n * np.sum(np.abs(c) ** 2), rtol=1e-12)
    assert np.allclose(core.weyl_compose(c, d), A, rtol=0, atol=1e-12)
    if d ** (3 * n) <= 3 ** 15:
        assert np.allclose(core.weyl_coeffs(A, d), c, rtol=0, atol=1e-13)


@pytest.mark.parametrize("d,n", [(3, 2), (5, 1), (3, 4)])
def test_weyl_single_operator_is_a_unit_vector(d, n):
    N = d ** n
    g = np.random.default_rng(d + n)
    for a, b in [(0, 0), (N - 1, 1), tuple(int(v) for v in g.integers(0, N, 2))]:
        W = kron.weyl_operator(d, kron._digits(a, d, n), kron._digits(b, d, n))
        c = core.weyl_coeffs_dft(W, d)
        e = np.zeros((N, N), dtype=np.complex128)
        e[a, b] = 1.0
        assert np.allclose(c, e, rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_weyl_d2_is_pauli_with_y_phase(n):
    # d = 2: X^x Z^z = (-i)^{#Y} sigma^t (XZ = -iY), so c_{x,z} = i^{#Y} w_t
    A = synth.general(n, seed=800 + n)
    w = oracle.coeffs_fwht(A)
    c = core.weyl_coeffs_dft(A, 2)
    N = 2 ** n
    x = np.repeat(np.arange(N), N)
    z = np.tile(np.arange(N), N)
    ny = np.array([bin(int(v)).count("1") for v in (x & z)])
    phase = np.array([1, 1j, -1, -1j])[ny % 4]             # i^{#Y}, exact
    want = phase * w[oracle.string_of_xz(x, z, n).astype(np.int64)]
    assert np.allclose(c.reshape(-1), want, rtol=0, atol=1e-14)
    Ai = synth.int_general(n, seed=810 + n)          # integers: d = 2 sums are exact
    wi = oracle.coeffs_fwht(Ai)
    ci = core.weyl_coeffs_dft(Ai, 2).reshape(-1)
    assert np.array_equal(ci, phase * wi[oracle.string_of_xz(x, z, n).astype(np.int64)])


@pytest.mark.parametrize("d,n", [(3, 3), (5, 2)])
def test_weyl_hermitian_symmetry(d, n):
    # W_{a,b} = omega^{-a.b} W_{-a,-b}^* (from Z X = omega X Z), so for
    # Hermitian A: conj(c_{a,b}) = d^-n tr(W_{a,b} A) = omega^{-a.b} c_{-a,-b}
    N = d ** n
    B = rand(N, 900 + d)
    A = (B + B.conj().T) / 2
    c = core.weyl_coeffs_dft(A, d)
    w = np.exp(2j * np.pi / d)
    for a in range(N):
        for b in range(N):
            assert abs(np.conj(c[a, b]) - w ** (-dot(a, b, d, n)) * c[neg(a, d, n), neg(b, d, n)]) <= 1e-14


def test_weyl_rows_of_chosen_shifts():
    # the per-shift entry, for complex128 and (gathered, widened) complex64
    # input, equals the rows of the full decomposition
    d, n = 3, 5
    A = rand(d ** n, 950)
    full = core.weyl_coeffs_dft(A, d)
    shifts = [0, 1, 7, d ** n - 1]
    assert np.array_equal(core.weyl_rows(A, d, shifts), full[shifts])
    A32 = A.astype(np.complex64)
    assert np.array_equal(core.weyl_rows(A32, d, shifts), core.weyl_coeffs_dft(A32.astype(np.complex128), d)[shifts])


def test_d3_unit_matrices_match_hand_derived_weights():
    # tests/golden/weyl_d3_unit_matrices.txt: the weights of the nine 3x3 unit
    # matrices, derived by hand from X|j> = |j+1>, Z|j> = w^j |j>
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "weyl_d3_unit_matrices.txt")

    def val(tok):
        if tok.lstrip("-") == "s":
            return (-1.0 if tok.startswith("-") else 1.0) * np.sqrt(3.0) / 6.0
        return float(tok) / 6.0

    seen = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        head, a, *cols = line.split("|")
        r, c = (int(v) for v in head.split())
        E = np.zeros((3, 3), dtype=np.complex128)
        E[r, c] = 1.0
        want = np.zeros((3, 3), dtype=np.complex128)
        for b, t in enumerate(cols):
            re, im = t.split()
            want[int(a), b] = val(re) + 1j * val(im)
        assert np.allclose(core.weyl_coeffs(E, 3), want, rtol=0, atol=1e-15), (r, c)
        assert np.allclose(kron.weyl_coeffs_kron(E, 3), want, rtol=0, atol=1e-15), (r, c)
        seen += 1
    assert seen == 9
