"""O0: Pauli decomposition by explicit Kronecker products (test infrastructure).

Eq. 1 builds sigma^t = sigma^{t_1} (x) ... (x) sigma^{t_n} with numpy.kron, the
first factor outermost (it indexes the most significant row/column bit, the
block partition of Eq. 3).  Eq. 2 then gives w_t = 2^-n tr(sigma^t A) by a
dense matrix product.  Exponential in memory and time: meant for n <= 4.
"""
import itertools

import numpy as np

# Sec. II.A: sigma^0..3 = I, X, Y, Z
SIGMA = (
    np.array([[1, 0], [0, 1]], dtype=np.complex128),
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
)


def pauli_string_matrix(t):
    """sigma^t for a sequence t = (t_1, ..., t_n) (Eq. 1)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for tj in t:
        m = np.kron(m, SIGMA[tj])
    return m


def _strings(n):
    # string order: base 4, t_1 most significant
    return itertools.product(range(4), repeat=n)


def coeffs_kron(A):
    """All 4^n weights of Eq. 2, string order, by dense products."""
    A = np.asarray(A, dtype=np.complex128)
    N = A.shape[0]
    n = N.bit_length() - 1
    out = np.empty(4 ** n, dtype=np.complex128)
    for s, t in enumerate(_strings(n)):
        out[s] = np.trace(pauli_string_matrix(t) @ A) / N
    return out


def compose_kron(w, n):
    """A = sum_t w_t sigma^t (Eq. 2, left side), w in string order."""
    N = 2 ** n
    A = np.zeros((N, N), dtype=np.complex128)
    for s, t in enumerate(_strings(n)):
        A += w[s] * pauli_string_matrix(t)
    return A


# ---------------------------------------------------------------- Weyl basis (qudits)

def weyl_single(d, a, b):
    """X^a Z^b for one qudit: X|j> = |j+1 mod d>, Z|j> = omega^j |j>, omega = e^(2 pi i/d)."""
    X = np.zeros((d, d), dtype=np.complex128)
    for j in range(d):
        X[(j + 1) % d, j] = 1.0
    Z = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
    return np.linalg.matrix_power(X, a) @ np.linalg.matrix_power(Z, b)


def weyl_operator(d, a_digits, b_digits):
    """The tensor product over qudits (qudit 1 outermost) of X^a_j Z^b_j."""
    m = np.ones((1, 1), dtype=np.complex128)
    for aj, bj in zip(a_digits, b_digits):
        m = np.kron(m, weyl_single(d, aj, bj))
    return m


def _digits(x, d, n):
    """Base-d digits of x, qudit 1 (most significant) first."""
    return [(x // d ** (n - 1 - j)) % d for j in range(n)]


def weyl_coeffs_kron(A, d):
    """c_{a,b} = d^-n tr(W_{a,b}^* A) for all a, b by dense products: (d^n, d^n) array [a, b]."""
    A = np.asarray(A, dtype=np.complex128)
    N = A.shape[0]
    n = int(round(np.log(N) / np.log(d)))
    out = np.empty((N, N), dtype=np.complex128)
    for a in range(N):
        for b in range(N):
            W = weyl_operator(d, _digits(a, d, n), _digits(b, d, n))
            out[a, b] = np.trace(W.conj().T @ A) / N
    return out


# ---------------------------------------------------------------- generalized Gell-Mann basis (qudits)

def gellmann_single(d, r, c):
    """The single-qudit generalized Gell-Mann element of label (r, c), a dense
    d x d matrix: the identity at (0, 0); the diagonal element
    sqrt(2 / (l (l+1))) diag(1, ..., 1, -l, 0, ..., 0) (l ones) at (l, l);
    E_rc + E_cr at (r, c) above the diagonal; -i E_cr + i E_rc at (r, c)
    below it (the antisymmetric element of the pair c < r)."""
    G = np.zeros((d, d), dtype=np.complex128)
    if r == 0 and c == 0:
        return np.eye(d, dtype=np.complex128)
    if r == c:
        diag = np.zeros(d)
        diag[:r] = 1.0
        diag[r] = -r
        return np.diag(diag * np.sqrt(2.0 / (r * (r + 1)))).astype(np.complex128)
    if r < c:
        G[r, c] = G[c, r] = 1.0
    else:
        j, k = c, r
        G[j, k] = -1j
        G[k, j] = 1j
    return G


def gellmann_operator(d, r_digits, c_digits):
    """The tensor product over qudits (qudit 1 outermost) of the single-qudit
    elements labelled (r_j, c_j)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for rj, cj in zip(r_digits, c_digits):
        m = np.kron(m, gellmann_single(d, rj, cj))
    return m


def gellmann_coeffs_kron(A, d):
    """g_(r,c) = tr(G_(r,c) A) / tr(G_(r,c)^2) for all labels by dense
    products: (d^n, d^n) array [r, c]."""
    A = np.asarray(A, dtype=np.complex128)
    N = A.shape[0]
    n = int(round(np.log(N) / np.log(d)))
    out = np.empty((N, N), dtype=np.complex128)
    for r in range(N):
        for c in range(N):
            G = gellmann_operator(d, _digits(r, d, n), _digits(c, d, n))
            out[r, c] = np.trace(G @ A) / np.trace(G @ G).real
    return out
