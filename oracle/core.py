"""ctypes front end of the C oracle ``tpd_oracle.c`` and of ``tpd_alg1.c`` (the
paper's recursive algorithm on the CPU) -- test infrastructure only.

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
_SRC_ALG1 = os.path.join(_HERE, "tpd_alg1.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build_library(force=False):
    """Compile tpd_oracle.c, tpd_alg1.c -> oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_ALG1))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, _SRC_ALG1, "-lm"]
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
            lib.oracle_compose.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_compose_fwht.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_tpd_alg1.argtypes = [dp, ctypes.c_int, dp]
            lib.oracle_tpd_alg2.argtypes = [dp, ctypes.c_int, dp]
            for f in (lib.oracle_coeffs, lib.oracle_coeffs_fwht, lib.oracle_coeffs_at,
                      lib.oracle_coeffs_xrows, lib.oracle_compose, lib.oracle_compose_fwht,
                      lib.oracle_tpd_alg1, lib.oracle_tpd_alg2):
                f.restype = ctypes.c_int
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


def tpd_alg1(A):
    """All 4^n weights by the paper's recursive algorithm (Alg. 1: CMWs of
    Eq. 4, recursion on nonzero CMWs), string order; single-threaded."""
    A, n = _square(A)
    out = np.empty(4 ** n, dtype=np.complex128)
    if _load().oracle_tpd_alg1(_dptr(A), n, _dptr(out)):
        raise RuntimeError("oracle_tpd_alg1 failed")
    return out


def tpd_alg2(A, overwrite=False):
    """All 4^n weights by the paper's iterative algorithm (Alg. 2: every CMW of
    a level split at once, in place, OpenMP over quads), string order.  With
    overwrite, A (complex128, contiguous) is used as the working array."""
    A, n = _square(A)
    W = A if overwrite else A.copy()
    out = np.empty(4 ** n, dtype=np.complex128)
    if _load().oracle_tpd_alg2(_dptr(W), n, _dptr(out)):
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
    Returns (count, N) complex array; string of (i, z) is string_of_xz(xs[i], z, n)."""
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
