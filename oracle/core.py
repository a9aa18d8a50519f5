"""ctypes front end of the C oracle ``tpd_oracle.c`` and of ``tpd_alg2.c`` (the
paper's iterative algorithm on the CPU) -- test infrastructure only.

The shared library is compiled with gcc into ``oracle/_build/`` on first use
(or by ``build_library()``), with -ffp-contract=off so that no sum in the
oracle is fused or reassociated.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpd_oracle.c")
_SRC_ALG2 = os.path.join(_HERE, "tpd_alg2.c")
_SRC_WEYL = os.path.join(_HERE, "tpd_weyl.c")
_SRC_GM = os.path.join(_HERE, "tpd_gellmann.c")
_SOURCES = (_SRC, _SRC_ALG2, _SRC_WEYL, _SRC_GM)
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force=False):
    """Compile tpd_oracle.c, tpd_alg2.c, tpd_weyl.c, tpd_gellmann.c -> oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(f) for f in _SOURCES)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp] + list(_SOURCES) + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_library())
            dp = ctypes.POINTER(ctypes.c_double)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            lib.oracle_coeffs.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_coeffs_fwht.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_coeffs_at.argtypes = [dp, ctypes.c_int, u64p, ctypes.c_int64, dp]
            lib.oracle_coeffs_xrows.argtypes = [dp, ctypes.c_int, u64p, ctypes.c_int64, dp]
            lib.oracle_coeffs_xdiags.argtypes = [dp, ctypes.c_int, u64p, ctypes.c_int64]
            lib.oracle_compose.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_compose_fwht.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_tpd_alg2.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int]
            for f in (lib.oracle_coeffs, lib.oracle_coeffs_fwht, lib.oracle_coeffs_at,
                      lib.oracle_coeffs_xrows, lib.oracle_coeffs_xdiags, lib.oracle_compose,
                      lib.oracle_compose_fwht,
                      lib.oracle_tpd_alg2):
                f.restype = ctypes.c_int
            lib.oracle_weyl_rows.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.c_int64, dp]
            lib.oracle_weyl_rows.restype = ctypes.c_int
            lib.oracle_weyl_diags.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
            lib.oracle_weyl_diags.restype = ctypes.c_int
            for f in (lib.oracle_weyl_coeffs, lib.oracle_weyl_coeffs_dft, lib.oracle_weyl_compose):
                f.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
                f.restype = ctypes.c_int
            for f in (lib.oracle_gm_coeffs, lib.oracle_gm_compose):
                f.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
                f.restype = ctypes.c_int
            i64p = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_gm_coeffs_at.argtypes = [dp, ctypes.c_int, ctypes.c_int, i64p, i64p, ctypes.c_int64, dp]
            lib.oracle_gm_coeffs_at.restype = ctypes.c_int
            lib.oracle_num_threads.argtypes = []
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u64ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _square(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    N = A.shape[0]
    if A.ndim != 2 or A.shape[1] != N or N & (N - 1):
        raise ValueError("A must be a 2^n x 2^n matrix")
    return A, N.bit_length() - 1


def num_threads():
    """OpenMP threads the oracle runs on."""
    return int(_load().oracle_num_threads())


def tpd_alg2(A, overwrite=False, threads=0):
    """All 4^n weights by the paper's iterative algorithm (Alg. 2: every CMW of
    a level split at once, in place, OpenMP over quads), string order.  With
    overwrite, A (complex128, contiguous) is used as the working array;
    threads: OpenMP threads (0: all)."""
    A, n = _square(A)
    W = A if overwrite else A.copy()
    out = np.empty(4 ** n, dtype=np.complex128)
    if _load().oracle_tpd_alg2(_dptr(W), n, _dptr(out), int(threads)):
        raise RuntimeError("oracle_tpd_alg2 failed")
    return out


def coeffs(A):
    """All 4^n weights by the signed-permutation trace, string order. O(8^n)."""
    A, n = _square(A)
    out = np.empty(4 ** n, dtype=np.complex128)
    if _load().oracle_coeffs(_dptr(A), n, _dptr(out)):
        raise RuntimeError("oracle_coeffs failed")
    return out


def coeffs_fwht(A):
    """All 4^n weights, string order, with the inner signed sums done by a
    Walsh-Hadamard transform per x-mask. O(n 4^n)."""
    A, n = _square(A)
    out = np.empty(4 ** n, dtype=np.complex128)
    if _load().oracle_coeffs_fwht(_dptr(A), n, _dptr(out)):
        raise RuntimeError("oracle_coeffs_fwht failed")
    return out


def coeffs_at(A, strings):
    """Weights of the given string indices (string order numbering). O(count 2^n)."""
    A, n = _square(A)
    s = np.ascontiguousarray(strings, dtype=np.uint64)
    out = np.empty(s.shape[0], dtype=np.complex128)
    if _load().oracle_coeffs_at(_dptr(A), n, _u64ptr(s), s.shape[0], _dptr(out)):
        raise RuntimeError("oracle_coeffs_at failed")
    return out


def coeffs_xrows(A, xs):
    """For each X-mask x in xs, the N weights w_(x,z), z = 0..N-1.
    Returns (count, N) complex array; string of (i, z) is string_of_xz(xs[i], z, n).
    A complex64 matrix is not widened as a whole: the entries A[r^x][r] of
    each requested x are gathered and widened to complex128 (exact)."""
    if isinstance(A, np.ndarray) and A.dtype == np.complex64 and A.ndim == 2:
        N = A.shape[0]
        if A.shape[1] != N or N & (N - 1):
            raise ValueError("A must be a 2^n x 2^n matrix")
        n = N.bit_length() - 1
        x = np.ascontiguousarray(xs, dtype=np.uint64)
        r = np.arange(N, dtype=np.int64)
        V = np.stack([A[r ^ int(xi), r].astype(np.complex128) for xi in x]) if x.size else \
            np.empty((0, N), dtype=np.complex128)
        V = np.ascontiguousarray(V)
        if _load().oracle_coeffs_xdiags(_dptr(V), n, _u64ptr(x), x.shape[0]):
            raise RuntimeError("oracle_coeffs_xdiags failed")
        return V
    A, n = _square(A)
    x = np.ascontiguousarray(xs, dtype=np.uint64)
    out = np.empty((x.shape[0], 2 ** n), dtype=np.complex128)
    if _load().oracle_coeffs_xrows(_dptr(A), n, _u64ptr(x), x.shape[0], _dptr(out)):
        raise RuntimeError("oracle_coeffs_xrows failed")
    return out


def compose(w, n):
    """A = sum_t w_t sigma^t (Eq. 2), w in string order. O(8^n)."""
    w = np.ascontiguousarray(w, dtype=np.complex128)
    if w.shape != (4 ** n,):
        raise ValueError("w must have 4^n entries")
    A = np.empty((2 ** n, 2 ** n), dtype=np.complex128)
    if _load().oracle_compose(_dptr(w), n, _dptr(A)):
        raise RuntimeError("oracle_compose failed")
    return A


def compose_fwht(w, n):
    """A = sum_t w_t sigma^t, w in string order, with the inner sums over z
    done by a Walsh-Hadamard transform per x-mask. O(n 4^n)."""
    w = np.ascontiguousarray(w, dtype=np.complex128)
    if w.shape != (4 ** n,):
        raise ValueError("w must have 4^n entries")
    A = np.empty((2 ** n, 2 ** n), dtype=np.complex128)
    if _load().oracle_compose_fwht(_dptr(w), n, _dptr(A)):
        raise RuntimeError("oracle_compose_fwht failed")
    return A


def grad_weighted_sq(A, weights):
    """Gradient of L(A) = sum_t w_t |c_t|^2, c = decomposition of A, in the
    convention dL/dRe + i dL/dIm.  c is linear in A with adjoint 2^-n times
    composition (the Pauli strings are Hermitian, Sec. II.A), and dL/dconj(c_t)
    = w_t c_t, so grad = 2 * 2^-n * sum_t w_t c_t sigma^t."""
    A, n = _square(A)
    c = coeffs_fwht(A)
    return compose_fwht(2.0 ** (1 - n) * np.asarray(weights, dtype=np.float64) * c, n)


def string_of_xz(x, z, n):
    """String index of the Pauli string with X-mask x and Z-mask z: at each
    qubit bit b, (x_b, z_b) = (0,0) I, (1,0) X, (1,1) Y, (0,1) Z."""
    x = np.asarray(x, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    s = np.zeros(np.broadcast(x, z).shape, dtype=np.uint64)
    code = np.array([0, 3, 1, 2], dtype=np.uint64)  # index = x_b*2 + z_b
    for b in range(n):
        xb = (x >> np.uint64(b)) & np.uint64(1)
        zb = (z >> np.uint64(b)) & np.uint64(1)
        s |= code[(xb * np.uint64(2) + zb).astype(np.int64)] << np.uint64(2 * b)
    return s


# ---------------------------------------------------------------- Weyl basis (qudits)

def _square_d(A, d):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    N = A.shape[0]
    n = 0
    while d ** n < N:
        n += 1
    if A.ndim != 2 or A.shape[1] != N or d ** n != N or n < 1:
        raise ValueError("A must be a d^n x d^n matrix")
    return A, n


def weyl_coeffs(A, d):
    """All d^2n weights c_{a,b} = d^-n tr(W_{a,b}^* A) in the Weyl
    (clock-and-shift) basis W_{a,b} = X^a Z^b, as a (d^n, d^n) array indexed
    [a, b] (see tpd_weyl.c for the digit convention).  O(d^3n)."""
    A, n = _square_d(A, d)
    N = d ** n
    out = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_weyl_coeffs(_dptr(A), n, d, _dptr(out)):
        raise RuntimeError("oracle_weyl_coeffs failed")
    return out


def weyl_coeffs_dft(A, d):
    """The same weights with the sum over c per shift a done as a
    tensor-product DFT over the base-d digits.  O(n d^(2n+1))."""
    A, n = _square_d(A, d)
    N = d ** n
    out = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_weyl_coeffs_dft(_dptr(A), n, d, _dptr(out)):
        raise RuntimeError("oracle_weyl_coeffs_dft failed")
    return out


def _digit_add(c, a, d, n):
    """digit-wise (c + a) mod d of base-d integers (c an array, a a scalar)"""
    out = np.zeros_like(c)
    p = 1
    for _ in range(n):
        out += ((c // p) % d + (a // p) % d) % d * p
        p *= d
    return out


def weyl_rows(A, d, shifts):
    """Weights c_{a,b}, b = 0..d^n-1, of the given shifts a: (count, d^n)
    array.  A matrix in another storage type (complex64) is not widened as a
    whole: the entries A[c + a][c] of each requested shift are gathered and
    widened to complex128 exactly."""
    N = A.shape[0]
    n = 0
    while d ** n < N:
        n += 1
    if A.ndim != 2 or A.shape[1] != N or d ** n != N:
        raise ValueError("A must be a d^n x d^n matrix")
    a_s = np.ascontiguousarray(shifts, dtype=np.int64)
    if np.any(a_s < 0) or np.any(a_s >= N):
        raise ValueError("shift out of range")
    if A.dtype == np.complex128 and A.flags.c_contiguous:
        out = np.empty((a_s.shape[0], N), dtype=np.complex128)
        if _load().oracle_weyl_rows(_dptr(A), n, d, a_s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    a_s.shape[0], _dptr(out)):
            raise RuntimeError("oracle_weyl_rows failed")
        return out
    c = np.arange(N, dtype=np.int64)
    V = np.ascontiguousarray(np.stack([A[_digit_add(c, int(a), d, n), c].astype(np.complex128) for a in a_s]))
    if _load().oracle_weyl_diags(_dptr(V), n, d, a_s.shape[0]):
        raise RuntimeError("oracle_weyl_diags failed")
    return V


def weyl_compose(C, d):
    """A = sum_{a,b} c_{a,b} W_{a,b} from the (d^n, d^n) weight array [a, b]."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    N = C.shape[0]
    n = 0
    while d ** n < N:
        n += 1
    if C.shape != (N, N) or d ** n != N:
        raise ValueError("C must be a d^n x d^n array of weights")
    A = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_weyl_compose(_dptr(C), n, d, _dptr(A)):
        raise RuntimeError("oracle_weyl_compose failed")
    return A


# ---------------------------------------------------------------- generalized Gell-Mann basis (qudits)

def gellmann_coeffs(A, d):
    """All d^2n coefficients g_(r,c) = tr(G_(r,c) A) / N_(r,c) in the
    generalized Gell-Mann basis, as a (d^n, d^n) array indexed [r, c] (the
    label of each basis element is a position of the d^n x d^n grid; see
    tpd_gellmann.c).  The trace over the nonzeros of every tensor product."""
    A, n = _square_d(A, d)
    N = d ** n
    out = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_gm_coeffs(_dptr(A), n, d, _dptr(out)):
        raise RuntimeError("oracle_gm_coeffs failed")
    return out


def gellmann_coeffs_at(A, d, rows, cols):
    """The coefficients of the labels (rows[i], cols[i]) (1-D array).  A matrix
    in another storage type (complex64) is widened to complex128 exactly."""
    A, n = _square_d(A, d)
    N = d ** n
    r = np.ascontiguousarray(rows, dtype=np.int64)
    c = np.ascontiguousarray(cols, dtype=np.int64)
    if r.shape != c.shape or r.ndim != 1:
        raise ValueError("rows and cols must be 1-D arrays of one length")
    if np.any(r < 0) or np.any(r >= N) or np.any(c < 0) or np.any(c >= N):
        raise ValueError("label out of range")
    out = np.empty(r.shape[0], dtype=np.complex128)
    i64 = ctypes.POINTER(ctypes.c_int64)
    if _load().oracle_gm_coeffs_at(_dptr(A), n, d, r.ctypes.data_as(i64), c.ctypes.data_as(i64), r.shape[0],
                                   _dptr(out)):
        raise RuntimeError("oracle_gm_coeffs_at failed")
    return out


def gellmann_compose(C, d):
    """A = sum_(r,c) g_(r,c) G_(r,c) from the (d^n, d^n) coefficient array."""
    C, n = _square_d(C, d)
    N = d ** n
    A = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_gm_compose(_dptr(C), n, d, _dptr(A)):
        raise RuntimeError("oracle_gm_compose failed")
    return A


def gellmann_norms(d, n):
    """N_(r,c) = tr(G_(r,c)^2) = prod over qudits of (d for the identity, 2
    otherwise), as a (d^n, d^n) float array [r, c]."""
    N = d ** n
    r = np.repeat(np.arange(N), N).reshape(N, N)
    c = np.tile(np.arange(N), N).reshape(N, N)
    out = np.ones((N, N))
    for _ in range(n):
        out *= np.where((r % d == 0) & (c % d == 0), float(d), 2.0)
        r, c = r // d, c // d
    return out
