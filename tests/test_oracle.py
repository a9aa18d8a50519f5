"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formula: each compares it with an
independent construction (the n=1 closed form of Eq. 4 typed by hand, dense
Kronecker products of Eq. 1, Parseval, reconstruction, Hermiticity, planted
Hamiltonians built from matrix elements, finite differences).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import kron
from paper_2310_13421_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _strings(n):
    return list(itertools.product(range(4), repeat=n))


def _count_y(t):
    return sum(1 for tj in t if tj == 2)


# ---------------------------------------------------------------- O0 itself

def test_kron_basis_is_orthonormal_hermitian_involutory():
    # Sec. II.A: Pauli strings are Hermitian, involutory, unitary and orthonormal
    # under <A,B> = 2^-n tr(A^* B).
    n = 2
    mats = [kron.pauli_string_matrix(t) for t in _strings(n)]
    N = 2 ** n
    for i, P in enumerate(mats):
        assert np.array_equal(P, P.conj().T)
        assert np.array_equal(P @ P, np.eye(N))
        for j, Q in enumerate(mats):
            ip = np.trace(P.conj().T @ Q) / N
            assert ip == (1.0 if i == j else 0.0)


def test_kron_first_factor_is_most_significant_bit():
    # Eq. 3: the first tensor factor selects the quadrant A11/A12/A21/A22.
    P = kron.pauli_string_matrix((1, 0))  # X (x) I
    N = 4
    for r in range(N):
        for c in range(N):
            assert P[r, c] == (1.0 if c == r ^ 2 else 0.0)


# ---------------------------------------------------------------- closed form, n = 1

def test_n1_unit_matrices_match_eq4_by_hand():
    rows = np.loadtxt(os.path.join(GOLDEN, "n1_unit_matrices.txt"))
    for row in rows:
        a, b = int(row[0]), int(row[1])
        E = np.zeros((2, 2), dtype=np.complex128)
        E[a, b] = 1.0
        want = row[2::2] + 1j * row[3::2]
        assert np.array_equal(oracle.coeffs(E), want)
        assert np.array_equal(oracle.coeffs_fwht(E), want)
        assert np.array_equal(kron.coeffs_kron(E), want)


# ---------------------------------------------------------------- brute force, n <= 3

@pytest.mark.parametrize("n", [1, 2, 3])
def test_signed_permutation_trace_matches_kronecker_random(n):
    A = synth.general(n, seed=100 + n)  # not Hermitian: a transposed or conjugated operand shows
    want = kron.coeffs_kron(A)
    for got in (oracle.coeffs(A), oracle.coeffs_fwht(A)):
        assert np.max(np.abs(got - want)) <= 1e-14 * np.max(np.abs(want))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_signed_permutation_trace_matches_kronecker_integer_exact(n):
    A = synth.int_general(n, seed=200 + n)
    want = kron.coeffs_kron(A)
    assert np.array_equal(oracle.coeffs(A), want)
    assert np.array_equal(oracle.coeffs_fwht(A), want)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_transposed_or_conjugated_operand_is_detected(n):
    # the pins above are sensitive to the plausible mistakes A^T and conj(A)
    A = synth.general(n, seed=300 + n)
    want = kron.coeffs_kron(A)
    assert np.max(np.abs(oracle.coeffs(A.T) - want)) > 1e-3
    assert np.max(np.abs(oracle.coeffs(A.conj()) - want)) > 1e-3


@pytest.mark.parametrize("n", [1, 2, 3])
def test_single_pauli_string_gives_unit_vector(n):
    # Sec. IV: decomposing one Pauli string sigma^t yields exactly e_t.
    for s, t in enumerate(_strings(n)):
        got = oracle.coeffs(kron.pauli_string_matrix(t))
        want = np.zeros(4 ** n, dtype=np.complex128)
        want[s] = 1.0
        assert np.array_equal(got, want)


def test_unit_matrix_is_identity_string():
    # Fig. 3 "unit matrix": only w_{0...0} = 1.
    for n in range(1, 7):
        got = oracle.coeffs_fwht(np.eye(2 ** n, dtype=np.complex128))
        assert got[0] == 1.0 and np.count_nonzero(got) == 1


# ---------------------------------------------------------------- O1 <-> O2 and sampled forms

@pytest.mark.parametrize("n", [4, 5, 6, 8])
def test_trace_and_walsh_hadamard_forms_agree(n):
    Ai = synth.int_general(n, seed=400 + n)
    assert np.array_equal(oracle.coeffs(Ai), oracle.coeffs_fwht(Ai))
    A = synth.hermitian(n, seed=410 + n)
    a, b = oracle.coeffs(A), oracle.coeffs_fwht(A)
    assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(a)


def test_sampled_and_xrow_forms_agree_with_full():
    n = 6
    A = synth.general(n, seed=500)
    full = oracle.coeffs(A)
    s = np.random.default_rng(1).integers(0, 4 ** n, size=300).astype(np.uint64)
    assert np.array_equal(oracle.coeffs_at(A, s), full[s.astype(np.int64)])
    xs = np.array([0, 1, 5, 63], dtype=np.uint64)
    rows = oracle.coeffs_xrows(A, xs)
    for i, x in enumerate(xs):
        z = np.arange(2 ** n, dtype=np.uint64)
        idx = oracle.string_of_xz(np.full_like(z, x), z, n).astype(np.int64)
        assert np.linalg.norm(rows[i] - full[idx]) <= 1e-14 * np.linalg.norm(full[idx])


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("n", [2, 5, 7])
def test_parseval(n):
    # orthonormal basis (Sec. II.A): ||A||_F^2 = 2^n sum |w_t|^2
    A = synth.general(n, seed=600 + n)
    w = oracle.coeffs_fwht(A)
    lhs = np.sum(np.abs(A) ** 2)
    rhs = 2 ** n * np.sum(np.abs(w) ** 2)
    assert abs(lhs - rhs) <= 1e-13 * lhs


@pytest.mark.parametrize("n", [1, 2, 3])
def test_compose_matches_kronecker_sum(n):
    w = synth.general(n + n, seed=700 + n).reshape(-1)[: 4 ** n]
    assert np.max(np.abs(oracle.compose(w, n) - kron.compose_kron(w, n))) <= 1e-14 * np.max(np.abs(w)) * 4 ** n


@pytest.mark.parametrize("n", [1, 3, 6])
def test_compose_forms_agree(n):
    wi = synth.int_general(n + n, seed=750 + n).reshape(-1)[: 4 ** n] / 4.0
    assert np.array_equal(oracle.compose(wi, n), oracle.compose_fwht(wi, n))
    w = synth.general(n + n, seed=760 + n).reshape(-1)[: 4 ** n]
    a, b = oracle.compose(w, n), oracle.compose_fwht(w, n)
    assert np.linalg.norm(a - b) <= 1e-14 * np.linalg.norm(a)


@pytest.mark.parametrize("n", [3, 6])
def test_reconstruction(n):
    # Eq. 2: A = sum_t w_t sigma^t; exact on integer inputs (dyadic weights)
    Ai = synth.int_general(n, seed=800 + n)
    assert np.array_equal(oracle.compose(oracle.coeffs(Ai), n), Ai)
    A = synth.hermitian(n, seed=810 + n)
    R = oracle.compose(oracle.coeffs(A), n)
    assert np.linalg.norm(R - A) <= 1e-14 * np.linalg.norm(A)


@pytest.mark.parametrize("n", [3, 6])
def test_hermitian_input_gives_real_weights(n):
    A = synth.hermitian(n, seed=900 + n)
    w = oracle.coeffs(A)
    assert np.max(np.abs(w.imag)) <= 1e-15 * np.max(np.abs(w)) * 2 ** n


@pytest.mark.parametrize("n", [3, 6])
def test_real_symmetric_odd_y_weights_vanish(n):
    # footnote of Sec. II.B / Sec. IV: real symmetric A has w_t = 0 for odd #Y
    A = synth.int_symmetric(n, seed=1000 + n)
    w = oracle.coeffs(A)
    for s, t in enumerate(_strings(n)):
        if _count_y(t) % 2 == 1:
            assert w[s] == 0.0
        else:
            assert w[s].imag == 0.0


# ---------------------------------------------------------------- planted Hamiltonians

@pytest.mark.parametrize("n", [2, 3, 4])
def test_heisenberg_generator_matches_kronecker(n):
    J, h = synth.heisenberg_params(n, seed=11)
    H = synth.heisenberg(n, J, h)
    K = np.zeros_like(H)
    for t, w in synth.heisenberg_terms(n, J, h).items():
        K += w * kron.pauli_string_matrix(t)
    assert np.array_equal(H, K)


@pytest.mark.parametrize("n", [2, 5, 7])
def test_heisenberg_device_writer_matches_dense_generator(n):
    torch = pytest.importorskip("torch")
    J, h = synth.heisenberg_params(n, seed=40 + n)
    H = torch.zeros((1 << n, 1 << n), dtype=torch.complex128)
    assert np.array_equal(synth.heisenberg_into(H, n, J, h).numpy(), synth.heisenberg(n, J, h))


@pytest.mark.parametrize("n", [3, 6, 8])
def test_heisenberg_terms_recovered_exactly(n):
    J, h = synth.heisenberg_params(n, seed=12 + n)
    w = oracle.coeffs_fwht(synth.heisenberg(n, J, h))
    want = np.zeros(4 ** n, dtype=np.complex128)
    for t, v in synth.heisenberg_terms(n, J, h).items():
        want[synth.string_index(t)] = v
    assert np.array_equal(w, want)
    assert np.count_nonzero(w) == 3 * (n - 1) + n


def test_tfim_eq7_terms_recovered_exactly():
    rows = np.loadtxt(os.path.join(GOLDEN, "tfim_first_level.txt"), ndmin=2)
    for n, J, g in rows:
        n = int(n)
        H = synth.tfim(n, J, g)
        if n <= 4:
            K = np.zeros_like(H)
            for t, v in synth.tfim_terms(n, J, g).items():
                K += v * kron.pauli_string_matrix(t)
            assert np.array_equal(H, K)
        w = oracle.coeffs(H)
        assert np.count_nonzero(w) == 2 * n - 1
        for t, v in synth.tfim_terms(n, J, g).items():
            assert w[synth.string_index(t)] == v


# ---------------------------------------------------------------- the paper's Alg. 2 on the CPU

@pytest.mark.parametrize("n", [1, 2, 3])
def test_alg2_matches_kronecker(n):
    A = synth.general(n, seed=340 + n)
    assert np.allclose(oracle.tpd_alg2(A), kron.coeffs_kron(A), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [1, 4, 6, 7, 9])
def test_alg2_integer_inputs_exact(n):
    Ai = synth.int_general(n, seed=350 + n)
    assert np.array_equal(oracle.tpd_alg2(Ai), oracle.coeffs(Ai) if n <= 6 else oracle.coeffs_fwht(Ai))


@pytest.mark.parametrize("n", [5, 8])
def test_alg2_random_within_rounding_bound(n):
    # every level rounds each output once (the 1/2 is exact) and is 2^-1/2 times
    # unitary: normwise error <= n u / (1 - n u) against the exact weights
    A = synth.general(n, seed=360 + n)
    want = oracle.coeffs_fwht(A)
    assert np.linalg.norm(oracle.tpd_alg2(A) - want) <= 2 * n * 2.0 ** -53 * np.linalg.norm(want)
    # the in-place form leaves the weights in the working array (RC layout)
    W = A.copy()
    oracle.tpd_alg2(W, overwrite=True)
    assert not np.array_equal(W, A)
    # the thread count does not change the result (each quad is computed once)
    assert np.array_equal(oracle.tpd_alg2(A, threads=1), oracle.tpd_alg2(A))


def test_alg2_prunes_zero_cmws_exactly():
    # planted Heisenberg chain (dyadic couplings): exactly the planted strings
    # are nonzero, with their exact values
    n = 8
    J, h = synth.heisenberg_params(n, seed=330)
    H = synth.heisenberg(n, J, h)
    want = np.zeros(4 ** n, dtype=np.complex128)
    for t, v in synth.heisenberg_terms(n, J, h).items():
        want[synth.string_index(t)] = v
    assert np.array_equal(oracle.tpd_alg2(H), want)
    # a diagonal matrix has only I/Z strings (x-mask 0)
    D = np.diag(synth.general(n, seed=331)[0]).astype(np.complex128)
    w = oracle.tpd_alg2(D)
    digits = np.arange(4 ** n)
    only_iz = np.ones(4 ** n, dtype=bool)
    for b in range(n):
        only_iz &= np.isin((digits >> (2 * b)) & 3, (0, 3))
    assert np.count_nonzero(w[~only_iz]) == 0
    assert np.allclose(w, oracle.coeffs_fwht(D), rtol=0, atol=1e-15)


# ---------------------------------------------------------------- gradient and adjoint

def test_adjoint_dot_product():
    # <D A, g> = <A, 2^-n C g> with <u,v> = sum conj(u) v: D^H = 2^-n C since
    # the Pauli strings are Hermitian (Sec. II.A)
    n = 4
    A = synth.general(n, seed=1200)
    g = synth.general(n + n, seed=1201).reshape(-1)[: 4 ** n]
    lhs = np.vdot(oracle.coeffs(A), g)
    rhs = np.vdot(A.reshape(-1), (2.0 ** -n) * oracle.compose(g, n).reshape(-1))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gradient_matches_central_differences():
    # L is quadratic in (Re A, Im A): central differences are exact up to rounding
    n = 3
    A = synth.hermitian(n, seed=1300)
    wts = synth.loss_weights(n, seed=1301)

    def loss(M):
        return float(np.sum(wts * np.abs(oracle.coeffs(M)) ** 2))

    G = oracle.grad_weighted_sq(A, wts)
    h = 1e-2
    rng = np.random.default_rng(5)
    for _ in range(16):
        i, j = rng.integers(0, 2 ** n, size=2)
        for unit, comp in ((1.0, "re"), (1j, "im")):
            Ap, Am = A.copy(), A.copy()
            Ap[i, j] += h * unit
            Am[i, j] -= h * unit
            fd = (loss(Ap) - loss(Am)) / (2 * h)
            an = G[i, j].real if comp == "re" else G[i, j].imag
            assert abs(fd - an) <= 1e-9 * max(1.0, abs(an))
