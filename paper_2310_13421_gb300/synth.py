"""Seeded synthetic inputs for the Pauli decomposition (shared by the CUDA path's
tests / benchmark and by the oracle's tests).

This module holds no step of the decomposition itself: it only draws matrices
and weights.  The spin Hamiltonians are written from their matrix elements in
the computational basis (diagonal Ising energies, spin-flip terms), not by
composing Pauli strings.

Conventions: A is row-major N x N, N = 2^n; qubit j = 1..n is row/column bit
n-j (qubit 1 most significant, the block partition of Eq. 3); a bit value s
gives the Z eigenvalue 1 - 2s.
"""
import concurrent.futures
import os

import numpy as np

DYADIC_BITS = 20  # couplings rounded to multiples of 2^-20 keep planted sums exact in fp64


def _rng(seed, *stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), *map(int, stream)])))


def _threads():
    return max(1, min(32, os.cpu_count() or 1))


def hermitian(n, seed, dtype=np.complex128):
    """A = (B + B^H)/2 with Re B, Im B i.i.d. N(0,1), 2^n x 2^n.  Exactly
    Hermitian in floating point: entry (i,j) and (j,i) are conjugate sums of
    the same pair.  B is drawn in fixed row blocks, one stream per block, and
    symmetrised in place tile by tile, so the bits do not depend on the thread
    count."""
    return hermitian_side(1 << n, seed, dtype)


def hermitian_side(N, seed, dtype=np.complex128):
    """hermitian() for any side N (e.g. d^n for n qudits of dimension d)."""
    rows_per = max(1, min(N, (1 << 22) // N))  # ~4M entries per stream
    A = np.empty((N, N), dtype=np.complex128)

    def draw(r0):
        g = _rng(seed, 1, r0)
        rows = min(rows_per, N - r0)
        A.real[r0:r0 + rows] = g.standard_normal((rows, N))
        A.imag[r0:r0 + rows] = g.standard_normal((rows, N))

    T = min(N, 512)  # symmetrisation tile

    def sym(ij):
        i, j = ij
        X = A[i:i + T, j:j + T]
        if i == j:
            X[...] = (X + X.T.conj()) * 0.5
        else:
            Y = A[j:j + T, i:i + T]
            S = (X + Y.T.conj()) * 0.5
            X[...] = S
            Y[...] = S.T.conj()

    with concurrent.futures.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(draw, range(0, N, rows_per)))
        list(ex.map(sym, [(i, j) for i in range(0, N, T) for j in range(i, N, T)]))
    if dtype == np.complex64:
        return A.astype(np.complex64)
    return A


def diag_dominant(n, seed, scale, dtype=np.complex128):
    """Hermitian matrix with a dominant diagonal: off-diagonal entries as in
    hermitian() (N(0,1) parts, conjugate-symmetric), diagonal real
    scale * N(0,1) -- strong local fields beside weak couplings, the case
    where elements of very different size share a tile."""
    A = hermitian(n, seed)
    g = _rng(seed, 3)
    A[np.diag_indices(1 << n)] = scale * g.standard_normal(1 << n)
    if dtype == np.complex64:
        return A.astype(np.complex64)
    return A


def general(n, seed):
    """Non-Hermitian complex matrix, Re/Im i.i.d. N(0,1) (for transposition checks)."""
    g = _rng(seed, 2)
    N = 1 << n
    return g.standard_normal((N, N)) + 1j * g.standard_normal((N, N))


def int_symmetric(n, seed, lo=-8, hi=8):
    """Real symmetric matrix with integer entries uniform in [lo, hi]."""
    g = _rng(seed, 3)
    N = 1 << n
    B = g.integers(lo, hi + 1, size=(N, N)).astype(np.float64)
    U = np.triu(B)
    S = U + np.triu(B, 1).T
    return S.astype(np.complex128)


def int_general(n, seed, lo=-8, hi=8):
    """Complex matrix with integer real and imaginary parts in [lo, hi]."""
    g = _rng(seed, 4)
    N = 1 << n
    re = g.integers(lo, hi + 1, size=(N, N)).astype(np.float64)
    im = g.integers(lo, hi + 1, size=(N, N)).astype(np.float64)
    return re + 1j * im


def dyadic(x, bits=DYADIC_BITS):
    """Round to the nearest multiple of 2^-bits (exact in fp64)."""
    return np.round(np.asarray(x, dtype=np.float64) * 2.0 ** bits) * 2.0 ** -bits


def heisenberg_params(n, seed, dyadic_bits=DYADIC_BITS):
    """Couplings J_j ~ U(-1,1) for the n-1 bonds and fields h_j ~ N(0,1) for the n sites.
    dyadic_bits=None leaves them unrounded."""
    g = _rng(seed, 5)
    J = g.uniform(-1.0, 1.0, size=n - 1)
    h = g.standard_normal(n)
    if dyadic_bits is not None:
        J, h = dyadic(J, dyadic_bits), dyadic(h, dyadic_bits)
    return J, h


def _z_values(n):
    """zv[j][r] = Z eigenvalue of qubit j+1 in basis state r (+1 for bit 0, -1 for bit 1)."""
    r = np.arange(1 << n, dtype=np.int64)
    return [1.0 - 2.0 * ((r >> (n - 1 - j)) & 1) for j in range(n)]


def heisenberg(n, J, h, dtype=np.complex128):
    """H = sum_j J_j (X_j X_j+1 + Y_j Y_j+1 + Z_j Z_j+1) + sum_j h_j Z_j, dense.
    Diagonal: sum_j J_j z_j z_j+1 + sum_j h_j z_j.  The XX+YY part maps
    |..01..> <-> |..10..> on the bond's two bits with amplitude 2 J_j."""
    N = 1 << n
    H = np.zeros((N, N), dtype=dtype)
    zv = _z_values(n)
    diag = np.zeros(N, dtype=np.float64)
    for j in range(n - 1):
        diag += J[j] * zv[j] * zv[j + 1]
    for j in range(n):
        diag += h[j] * zv[j]
    idx = np.arange(N, dtype=np.int64)
    H[idx, idx] = diag
    for j in range(n - 1):
        b_hi, b_lo = n - 1 - j, n - 2 - j
        s_hi = (idx >> b_hi) & 1
        s_lo = (idx >> b_lo) & 1
        flip = s_hi != s_lo
        r = idx[flip]
        rp = r ^ ((1 << b_hi) | (1 << b_lo))
        H[rp, r] = 2.0 * J[j]
    return H


def heisenberg_into(H, n, J, h):
    """Write the chain of heisenberg(n, J, h) into the zero torch tensor H
    (N x N complex, any device) without building it on the host: the same
    entries, the diagonal accumulated in the same order.  For sizes whose
    dense host copy would not fit (n = 16: 64 GB)."""
    import torch
    N = 1 << n
    dev = H.device
    idx = torch.arange(N, device=dev, dtype=torch.int64)
    z = [1.0 - 2.0 * ((idx >> (n - 1 - j)) & 1).to(torch.float64) for j in range(n)]
    diag = torch.zeros(N, dtype=torch.float64, device=dev)
    for j in range(n - 1):
        diag += float(J[j]) * z[j] * z[j + 1]
    for j in range(n):
        diag += float(h[j]) * z[j]
    flat = H.view(-1)
    flat[idx * (N + 1)] = diag.to(H.dtype)
    for j in range(n - 1):
        b_hi, b_lo = n - 1 - j, n - 2 - j
        flip = ((idx >> b_hi) & 1) != ((idx >> b_lo) & 1)
        r = idx[flip]
        rp = r ^ ((1 << b_hi) | (1 << b_lo))
        flat[rp * N + r] = 2.0 * float(J[j])
    return H


def heisenberg_terms(n, J, h):
    """The planted decomposition: {quaternary string tuple: weight}."""
    terms = {}
    for j in range(n - 1):
        for p in (1, 2, 3):
            t = [0] * n
            t[j] = t[j + 1] = p
            terms[tuple(t)] = J[j]
    for j in range(n):
        t = [0] * n
        t[j] = 3
        terms[tuple(t)] = terms.get(tuple(t), 0.0) + h[j]
    return terms


def tfim(n, J, g_field, dtype=np.complex128):
    """Eq. 7: H = -J (sum_i Z_i Z_i+1 + g sum_j X_j), dense.
    Diagonal -J sum z_i z_i+1; X_j flips bit n-j with amplitude -J g."""
    N = 1 << n
    H = np.zeros((N, N), dtype=dtype)
    zv = _z_values(n)
    diag = np.zeros(N, dtype=np.float64)
    for i in range(n - 1):
        diag += zv[i] * zv[i + 1]
    idx = np.arange(N, dtype=np.int64)
    H[idx, idx] = -J * diag
    for j in range(n):
        H[idx ^ (1 << (n - 1 - j)), idx] = -J * g_field
    return H


def tfim_terms(n, J, g_field):
    terms = {}
    for i in range(n - 1):
        t = [0] * n
        t[i] = t[i + 1] = 3
        terms[tuple(t)] = -J
    for j in range(n):
        t = [0] * n
        t[j] = 1
        terms[tuple(t)] = -J * g_field
    return terms


def string_index(t):
    """String-order index of the quaternary tuple t (t_1 most significant)."""
    s = 0
    for tj in t:
        s = 4 * s + int(tj)
    return s


def loss_weights(n, seed):
    """w_t ~ U(0,1) for the weighted loss L = sum_t w_t |c_t|^2."""
    return _rng(seed, 6).uniform(0.0, 1.0, size=4 ** n)


def batch_sizes(count, seed, n_lo=3, n_hi=10):
    """Qubit counts n_i uniform on {n_lo..n_hi}."""
    return _rng(seed, 7).integers(n_lo, n_hi + 1, size=count)
