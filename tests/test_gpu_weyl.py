"""GPU: decomposition in the Weyl (clock-and-shift) basis of qudits (the
tensorized basis Sec. V names for the method), through the C ABI, against the
Weyl oracle.

Tolerance.  Each qudit level maps every d x d block by d^-1 times a unitary
(the DFT along each cyclic diagonal), with a few roundings per output: for
d = 3 the written-out 3-point DFT rounds s = x1 + x2, u = x1 - x2, m, h u and
the final sum (five roundings, plus sqrt(3)/2 rounded once) and the 1/3 scale
once more; for d = 2, 4, 5 the plain DFT adds at most d - 1 rounded products.
So each level adds at most c_d u relative error in the 2-norm with c_d <= 16,
and n levels give ||c^ - c|| <= 16 n u ||c|| (u = 2^-53 complex128, 2^-24
complex64); the oracle's own fp64 error is far below it.  The complex128 block
fixed point (d = 2, 3, 4) rounds each output once per level (RNE) after sums
that are exact on its class's grid, up to sqrt(3) and the third rounded on
that grid (2^-59 of the class's largest element), so it meets the same bound
-- per weight relative to its own shift's magnitude, since classes never mix
shifts.  For d = 2 every operation is exact on integer inputs (twiddles +-1,
scale 1/2): bit-exact in both arithmetics.
"""
import numpy as np
import pytest

import oracle
from oracle import core
from paper_2310_13421_gb300 import synth
from _helpers import U32, U64, rel_err

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


def digit_add(x, y, d, n):
    out, p = np.zeros_like(x), 1
    for _ in range(n):
        out += ((x // p) % d + (y // p) % d) % d * p
        p *= d
    return out


def to_ab(W, d, n):
    """[a, b] array from a result in the kernel's layout: weight (a, b) at row
    digits b, column digits a + b mod d."""
    N = d ** n
    a = np.repeat(np.arange(N), N)
    b = np.tile(np.arange(N), N)
    return W[b, digit_add(a, b, d, n)].reshape(N, N)


def rand(N, seed, hermitian=False):
    g = np.random.default_rng(seed)
    A = g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))
    return (A + A.conj().T) / 2 if hermitian else A


@pytest.mark.parametrize("d,n", [(3, 1), (3, 2), (3, 3), (3, 4), (3, 5), (3, 6), (2, 5), (4, 3), (5, 2), (5, 3)])
@pytest.mark.parametrize("dtype,precision", [("c128", "fixed"), ("c128", "plain"), ("c64", None)])
def test_weyl_matches_oracle(tpd, d, n, dtype, precision):
    N = d ** n
    A = rand(N, 1000 + 10 * d + n)
    tt, u = (torch.complex128, U64) if dtype == "c128" else (torch.complex64, U32)
    if dtype == "c64":
        A = A.astype(np.complex64)
    if precision == "fixed" and d == 5:
        precision = None                      # d = 5: IEEE fp64 (the default)
    want = core.weyl_coeffs_dft(A.astype(np.complex128), d)
    got = to_ab(host(tpd.weyl_decompose(gpu(A, tt), d, precision=precision)).astype(np.complex128), d, n)
    e = rel_err(got, want)
    assert e <= 16 * n * u, "d=%d n=%d %s: %.3e" % (d, n, dtype, e)
    m = np.max(np.abs(got - want)) / np.max(np.abs(want))
    assert m <= 16 * n * u


@pytest.mark.parametrize("d", [2, 3, 4])
def test_weyl_fixed_point_per_class_accuracy(tpd, d):
    # block fixed point, complex128: each class (the d elements one DFT adds)
    # has its own binary point, so a weak diagonal beside strong ones keeps
    # fp64-class accuracy.  A strong diagonal (1e8) and weak off-diagonal
    # entries (1e-4) in every block: the shifts a != 0 carry only weak
    # entries, and their weights are checked per weight, relative to their
    # own shift's magnitude, against the oracle.
    n = {2: 6, 3: 4, 4: 3}[d]
    N = d ** n
    g = np.random.default_rng(1400 + d)
    A = 1e-4 * (g.standard_normal((N, N)) + 1j * g.standard_normal((N, N)))
    A[np.arange(N), np.arange(N)] = 1e8 * g.standard_normal(N)
    want = core.weyl_coeffs_dft(A, d)
    got = to_ab(host(tpd.weyl_decompose(gpu(A), d, precision="fixed")), d, n)
    for a in range(1, N):
        scale = np.max(np.abs(want[a]))
        assert np.max(np.abs(got[a] - want[a])) <= 16 * n * U64 * scale, "shift %d" % a


def test_weyl_fixed_point_non_finite_classes_follow_ieee(tpd):
    # a class meeting Inf / NaN takes the IEEE DFT: the non-finite weights
    # are where the fp64 form puts them, the finite ones agree to rounding
    d, n = 3, 4
    N = d ** n
    A = rand(N, 1500)
    A[7, 11] = np.inf
    A[40, 2] = complex(0.0, np.nan)
    fx = host(tpd.weyl_decompose(gpu(A), d, precision="fixed"))
    fp = host(tpd.weyl_decompose(gpu(A), d, precision="plain"))
    assert np.array_equal(np.isnan(fx), np.isnan(fp)) and np.array_equal(np.isinf(fx), np.isinf(fp))
    fin = np.isfinite(fx) & np.isfinite(fp)
    assert fin.sum() > 0 and rel_err(fx[fin], fp[fin]) <= 32 * n * U64


@pytest.mark.parametrize("n", [1, 4, 7])
def test_weyl_d2_is_the_pauli_decomposition(tpd, n):
    # d = 2: the Pauli RC layout, c = i^{#Y} w; integer inputs bit-exact
    A = synth.int_general(n, seed=1100 + n)
    got = host(tpd.weyl_decompose(gpu(A), 2)).reshape(-1)
    pauli = host(tpd.decompose(gpu(A), precision="plain")).reshape(-1)
    N = 2 ** n
    pos = np.arange(N * N)
    r, c = pos // N, pos % N
    ny = np.array([bin(int(v)).count("1") for v in (r & ~c & (N - 1))])      # Y at (r, c) = (1, 0)
    phase = np.array([1, 1j, -1, -1j])[ny % 4]
    assert np.array_equal(got, phase * pauli)
    want = core.weyl_coeffs_dft(A, 2)
    assert np.array_equal(to_ab(got.reshape(N, N), 2, n), want)


@pytest.mark.parametrize("d,n", [(3, 4), (5, 2)])
def test_weyl_compose_inverts_and_is_the_adjoint(tpd, d, n):
    N = d ** n
    A = rand(N, 1200 + d)
    C = tpd.weyl_decompose(gpu(A), d)
    assert rel_err(host(tpd.weyl_compose(C, d)), A) <= 32 * n * U64
    # <D A, G> = <A, d^-n C G> for a random G (both in the kernel's layout):
    # W_{a,b} is unitary, so the decomposition's adjoint is d^-n times the
    # composition
    G = rand(N, 1210 + d)
    lhs = np.vdot(host(C), G)
    rhs = np.vdot(A, host(tpd.weyl_compose(gpu(G), d, scale=float(d) ** -n)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def neg(x, d, n):
    out, p = 0, 1
    for _ in range(n):
        out += ((-((x // p) % d)) % d) * p
        p *= d
    return out


def dot(x, y, d, n):
    s, p = 0, 1
    for _ in range(n):
        s += ((x // p) % d) * ((y // p) % d)
        p *= d
    return s % d


def test_weyl_sampled_rows_and_hermitian_symmetry_n8(tpd):
    # n = 8 qutrits (6561 x 6561): sampled shifts against the oracle, and the
    # conjugation symmetry of a Hermitian input, conj(c_{a,b}) =
    # omega^{-a.b} c_{-a,-b} (from Z X = omega X Z)
    d, n = 3, 8
    N = d ** n
    A = rand(N, 1300, hermitian=True)
    W = host(tpd.weyl_decompose(gpu(A), d))
    rng = np.random.default_rng(3)
    shifts = [0, 1, N - 1] + [int(v) for v in rng.integers(0, N, 5)]
    want = core.weyl_rows(A, d, shifts)
    b = np.arange(N)
    got = np.stack([W[b, digit_add(b, np.full(N, a), d, n)] for a in shifts])
    assert rel_err(got, want) <= 16 * n * U64
    omega = np.exp(2j * np.pi / d)
    for a in shifts[3:]:
        for bb in rng.integers(0, N, 20):
            bb = int(bb)
            c_ab = W[bb, digit_add(np.array([bb]), np.array([a]), d, n)[0]]
            na, nb = neg(a, d, n), neg(bb, d, n)
            c_neg = W[nb, digit_add(np.array([nb]), np.array([na]), d, n)[0]]
            ph = omega ** (-dot(a, bb, d, n))
            assert abs(np.conj(c_ab) - ph * c_neg) <= 64 * n * U64 * np.max(np.abs(want))
