"""GPU: decomposition in the generalized Gell-Mann basis of qudits (the other
tensorized basis Sec. V names for the method), through the C ABI, against the
Gell-Mann oracle.

Tolerance.  With N_(r,c) = tr(G_(r,c)^2), the weighted norm
||g||_N = sqrt(sum N_(r,c) |g_(r,c)|^2) equals ||A||_F (Parseval), and each
qudit level is an isometry from the weighted norm of the levels done so far
to that of one more level.  A level rounds each output a few times: the
off-diagonal pairs twice (sum, halving: exact), the diagonal ones at most
d + 2 times (running sum, l x_ll, difference, factor c_l / 2) and the
identity's d times, each relative to the block's own entries.  So a level adds
at most c_d u ||x|| with c_d <= 16 for d <= 5, and n levels give
||g^ - g||_N <= 16 n u ||g||_N (u = 2^-53 complex128, 2^-24 complex64); the
oracle's own fp64 error is far below it.  For d = 2 every operation is exact
on integer inputs: bit-exact, and equal to the Pauli decomposition.  Real and
imaginary parts see the same operations, so conjugate blocks stay exact
conjugates: Hermitian inputs give exactly real coefficients.
"""
import numpy as np
import pytest

from oracle import core
from paper_2310_13421_gb300 import synth
from _helpers import U32, U64

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


def rand(N, seed, hermitian=False):
    g = np.random.default_rng(seed)
    A = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    return (A + A.conj().T) / 2 if hermitian else A


def norms_at(d, n, r, c):
    """N_(r,c) of the labels (r[i], c[i])"""
    r, c = np.array(r, dtype=np.int64), np.array(c, dtype=np.int64)
    out = np.ones(r.shape)
    for _ in range(n):
        out *= np.where((r % d == 0) & (c % d == 0), float(d), 2.0)
        r, c = r // d, c // d
    return out


def wrel(got, want, Nt):
    """relative error in the weighted norm ||x||_N = sqrt(sum N |x|^2)"""
    w = np.sqrt(Nt)
    return np.linalg.norm((w * (got - want)).reshape(-1)) / np.linalg.norm((w * want).reshape(-1))


@pytest.mark.parametrize("d,n", [(2, 5), (3, 1), (3, 2), (3, 4), (3, 6), (4, 3), (5, 2), (5, 3)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gellmann_matches_oracle(tpd, d, n, dtype):
    N = d ** n
    A = rand(N, 2000 + 10 * d + n)
    tt, u = (torch.complex128, U64) if dtype == "c128" else (torch.complex64, U32)
    if dtype == "c64":
        A = A.astype(np.complex64)
    want = core.gellmann_coeffs(A.astype(np.complex128), d)
    got = host(tpd.gellmann_decompose(gpu(A, tt), d)).astype(np.complex128)
    Nt = core.gellmann_norms(d, n)
    e = wrel(got, want, Nt)
    assert e <= 16 * n * u, "d=%d n=%d %s: %.3e" % (d, n, dtype, e)
    m = np.max(np.sqrt(Nt) * np.abs(got - want)) / np.linalg.norm(A)
    assert m <= 16 * n * u


@pytest.mark.parametrize("d,n", [(3, 5), (4, 3), (5, 2), (2, 6)])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_gellmann_hermitian_input_gives_exactly_real_coefficients(tpd, d, n, dtype):
    A = rand(d ** n, 2100 + d, hermitian=True)
    g = host(tpd.gellmann_decompose(gpu(A, dtype), d))
    assert np.all(g.imag == 0), "largest imaginary part %.3e" % np.max(np.abs(g.imag))
    assert np.max(np.abs(g.real)) > 0


@pytest.mark.parametrize("n", [1, 4, 7])
def test_gellmann_d2_is_the_pauli_decomposition(tpd, n):
    # d = 2: I, X, Y, Z at (0,0), (0,1), (1,0), (1,1), each of norm 2 -- the
    # Pauli RC layout and weights; integer inputs bit-exact
    A = synth.int_general(n, seed=2200 + n)
    got = host(tpd.gellmann_decompose(gpu(A), 2))
    assert np.array_equal(got, host(tpd.decompose(gpu(A), precision="plain")))
    assert np.array_equal(got, core.gellmann_coeffs(A, 2))
    B = synth.general(n, seed=2210 + n)
    gb = host(tpd.gellmann_decompose(gpu(B), 2))
    pb = host(tpd.decompose(gpu(B), precision="plain"))
    assert np.linalg.norm(gb - pb) <= 4 * n * U64 * np.linalg.norm(pb)


@pytest.mark.parametrize("d,n", [(3, 4), (5, 2), (4, 3)])
def test_gellmann_compose_inverts_and_gives_the_adjoint(tpd, d, n):
    N = d ** n
    A = rand(N, 2300 + d)
    C = tpd.gellmann_decompose(gpu(A), d)
    back = host(tpd.gellmann_compose(C, d))
    assert np.linalg.norm(back - A) <= 32 * n * U64 * np.linalg.norm(A)
    # against the oracle's composition of the same coefficients
    Cw = host(C)
    assert np.linalg.norm(host(tpd.gellmann_compose(gpu(Cw), d)) - core.gellmann_compose(Cw, d)) <= \
        32 * n * U64 * np.linalg.norm(A)
    # <D A, G> = <A, compose(G / N)> for a random G: the decomposition's
    # adjoint is the composition of the coefficients divided by their norms
    Nt = core.gellmann_norms(d, n)
    G = rand(N, 2310 + d)
    lhs = np.vdot(Cw, G)
    rhs = np.vdot(A, host(tpd.gellmann_compose(gpu(G / Nt), d)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # scale on the composition
    s = host(tpd.gellmann_compose(gpu(Cw), d, scale=0.375))
    assert np.linalg.norm(s - 0.375 * back) <= 4 * U64 * np.linalg.norm(back)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_gellmann_sampled_labels_n8(tpd, dtype):
    # n = 8 qutrits (6561 x 6561): sampled labels against the oracle, and
    # exactly real coefficients of a Hermitian input
    d, n = 3, 8
    N = d ** n
    A = rand(N, 2400, hermitian=True)
    tt, u = (torch.complex128, U64) if dtype == "c128" else (torch.complex64, U32)
    if dtype == "c64":
        A = A.astype(np.complex64)
    W = host(tpd.gellmann_decompose(gpu(A, tt), d))
    assert np.all(W.imag == 0)
    rng = np.random.default_rng(5)
    rows = np.concatenate([[0, N - 1, 0, N - 1, 1], rng.integers(0, N, 200)])
    cols = np.concatenate([[0, N - 1, N - 1, 0, 1], rng.integers(0, N, 200)])
    # and labels on the diagonal (identity / diagonal elements on every qudit)
    diag = rng.integers(0, N, 40)
    rows, cols = np.concatenate([rows, diag]), np.concatenate([cols, diag])
    want = core.gellmann_coeffs_at(A.astype(np.complex128), d, rows, cols)
    got = W[rows, cols].astype(np.complex128)
    Nt = norms_at(d, n, rows, cols)
    assert wrel(got, want, Nt) <= 16 * n * u
