"""ctypes binding of libtpd.so: the C ABI of include/tpd.h, same names, argument
marshalling only.  Loading fails loudly when the library is missing; there is
no fallback implementation."""
import ctypes
import os
import threading

from .buildlib import LIB

TPD_OK = 0
TPD_ERR_INVALID_ARG = 1
TPD_ERR_UNSUPPORTED = 2
TPD_ERR_MISALIGNED = 3
TPD_ERR_WORKSPACE = 4
TPD_ERR_CUDA = 5
TPD_ERR_TIMEOUT = 6

TPD_C128 = 0
TPD_C64 = 1

TPD_PREC_DEFAULT = 0
TPD_PREC_PLAIN = 1
TPD_PREC_COMPENSATED = 2
TPD_PREC_FIXED = 3

# every symbol include/tpd.h declares
SYMBOLS = (
    "tpd_options_init", "tpd_workspace_size", "tpd_decompose", "tpd_compose", "tpd_decompose_host",
    "tpd_batched_workspace_size", "tpd_decompose_batched", "tpd_compose_batched",
    "tpd_plan_describe", "tpd_status_string", "tpd_version", "tpd_decompose_noalloc",
    "tpd_tune_set", "tpd_tune_clear", "tpd_batch_status", "tpd_test_hold_batch_waits",
    "tpd_convert_layout", "tpd_sum_squares", "tpd_partial_workspace_size", "tpd_partial_prepare",
    "tpd_decompose_partial", "tpd_nonzero_workspace_size", "tpd_nonzero_list", "tpd_sparse_workspace_size",
    "tpd_decompose_coo", "tpd_weyl_decompose", "tpd_weyl_compose", "tpd_gellmann_decompose",
    "tpd_gellmann_compose",
)

# size of the library's own scratch array used by tpd_decompose_noalloc
TPD_NOALLOC_SCRATCH_BYTES = 64 << 20
# device workspace of tpd_sum_squares
TPD_SUMSQ_WORKSPACE_BYTES = 8192


class tpd_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("skip_zero", ctypes.c_int),
                ("tile_bits", ctypes.c_int), ("max_levels", ctypes.c_int), ("variant", ctypes.c_int),
                ("pass_events", ctypes.POINTER(ctypes.c_void_p)), ("num_events", ctypes.c_int),
                ("l2_chunk_mb", ctypes.c_int)]


class TPDError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s: %s" % (what, status_string(status)))
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path=None):
    """Load libtpd.so (built by paper_2310_13421_gb300.build.build())."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB
        if not os.path.exists(p):
            raise RuntimeError("libtpd.so not found at %s: run paper_2310_13421_gb300.build.build() "
                               "(the CUDA library is required; there is no CPU fallback)" % p)
        lib = ctypes.CDLL(p)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        op = ctypes.POINTER(tpd_options)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.tpd_options_init.argtypes = [op]
        lib.tpd_options_init.restype = None
        lib.tpd_workspace_size.argtypes = [i, i, op]
        lib.tpd_workspace_size.restype = sz
        lib.tpd_decompose.argtypes = [vp, i, i, op, vp, sz, vp]
        lib.tpd_decompose.restype = i
        lib.tpd_compose.argtypes = [vp, i, i, ctypes.c_double, op, vp, sz, vp]
        lib.tpd_compose.restype = i
        lib.tpd_tune_set.argtypes = [i, i, i, op]
        lib.tpd_tune_set.restype = i
        lib.tpd_tune_clear.argtypes = []
        lib.tpd_tune_clear.restype = None
        lib.tpd_partial_workspace_size.argtypes = [i, i, op, sz]
        lib.tpd_partial_workspace_size.restype = sz
        lib.tpd_partial_prepare.argtypes = [i, i, op, ctypes.POINTER(ctypes.c_ulonglong), sz, vp, sz, vp]
        lib.tpd_partial_prepare.restype = i
        lib.tpd_decompose_partial.argtypes = [vp, i, i, op, sz, vp, sz, vp, vp]
        lib.tpd_decompose_partial.restype = i
        lib.tpd_sparse_workspace_size.argtypes = [sz]
        lib.tpd_sparse_workspace_size.restype = sz
        lib.tpd_decompose_coo.argtypes = [vp, vp, vp, sz, i, i, sz, vp, vp, sz, vp, vp, vp, sz, vp]
        lib.tpd_decompose_coo.restype = i
        lib.tpd_nonzero_workspace_size.argtypes = [i]
        lib.tpd_nonzero_workspace_size.restype = sz
        lib.tpd_nonzero_list.argtypes = [vp, i, i, ctypes.c_double, vp, vp, sz, vp, vp, sz, vp]
        lib.tpd_nonzero_list.restype = i
        lib.tpd_weyl_decompose.argtypes = [vp, i, i, i, op, vp]
        lib.tpd_weyl_decompose.restype = i
        lib.tpd_weyl_compose.argtypes = [vp, i, i, i, ctypes.c_double, op, vp]
        lib.tpd_weyl_compose.restype = i
        lib.tpd_gellmann_decompose.argtypes = [vp, i, i, i, op, vp]
        lib.tpd_gellmann_decompose.restype = i
        lib.tpd_gellmann_compose.argtypes = [vp, i, i, i, ctypes.c_double, op, vp]
        lib.tpd_gellmann_compose.restype = i
        lib.tpd_convert_layout.argtypes = [vp, vp, i, i, i, vp]
        lib.tpd_convert_layout.restype = i
        lib.tpd_sum_squares.argtypes = [vp, sz, i, vp, vp, sz, vp]
        lib.tpd_sum_squares.restype = i
        lib.tpd_batch_status.argtypes = [vp, vp]
        lib.tpd_batch_status.restype = i
        lib.tpd_test_hold_batch_waits.argtypes = [i]
        lib.tpd_test_hold_batch_waits.restype = None
        lib.tpd_decompose_noalloc.argtypes = [vp, i, i, op, vp]
        lib.tpd_decompose_noalloc.restype = i
        lib.tpd_decompose_host.argtypes = [vp, vp, vp, i, i, op, vp, sz, vp]
        lib.tpd_decompose_host.restype = i
        lib.tpd_batched_workspace_size.argtypes = [ip, i, i, op]
        lib.tpd_batched_workspace_size.restype = sz
        lib.tpd_decompose_batched.argtypes = [vp, vp, ip, i, i, op, vp, sz, vp]
        lib.tpd_decompose_batched.restype = i
        lib.tpd_compose_batched.argtypes = [vp, vp, ip, i, i, i, op, vp, sz, vp]
        lib.tpd_compose_batched.restype = i
        lib.tpd_plan_describe.argtypes = [i, i, op, ctypes.c_char_p, sz]
        lib.tpd_plan_describe.restype = i
        lib.tpd_status_string.argtypes = [i]
        lib.tpd_status_string.restype = ctypes.c_char_p
        lib.tpd_version.argtypes = []
        lib.tpd_version.restype = i
        _lib = lib
        return lib


def options(precision=TPD_PREC_DEFAULT, skip_zero=False, tile_bits=0, max_levels=0, variant=0, pass_events=None,
            l2_chunk_mb=0):
    """tpd_options; pass_events: sequence of cudaEvent_t handles (ints) for the profiling hook."""
    o = tpd_options(int(precision), int(bool(skip_zero)), int(tile_bits), int(max_levels), int(variant), None, 0,
                    int(l2_chunk_mb))
    if pass_events:
        arr = (ctypes.c_void_p * len(pass_events))(*[int(e) for e in pass_events])
        o.pass_events = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
        o.num_events = len(pass_events)
        o._keep = arr  # keep the array alive with the struct
    return o


def _opt(opt):
    return ctypes.byref(opt) if opt is not None else None


def status_string(status):
    return load().tpd_status_string(int(status)).decode()


def tpd_workspace_size(n, dtype, opt=None):
    return int(load().tpd_workspace_size(n, dtype, _opt(opt)))


def tpd_decompose(A_ptr, n, dtype, opt=None, workspace=0, workspace_bytes=0, stream=0):
    return int(load().tpd_decompose(A_ptr, n, dtype, _opt(opt), workspace or None, workspace_bytes,
                                    stream or None))


def tpd_compose(C_ptr, n, dtype, scale, opt=None, workspace=0, workspace_bytes=0, stream=0):
    return int(load().tpd_compose(C_ptr, n, dtype, float(scale), _opt(opt), workspace or None,
                                  workspace_bytes, stream or None))


def tpd_tune_set(n, dtype, precision, tuned=None):
    return int(load().tpd_tune_set(n, dtype, precision, _opt(tuned)))


def tpd_tune_clear():
    load().tpd_tune_clear()


def tpd_partial_workspace_size(n, dtype, opt, count):
    return int(load().tpd_partial_workspace_size(n, dtype, _opt(opt), count))


def tpd_partial_prepare(n, dtype, opt, strings, workspace, workspace_bytes, stream=0):
    """strings: sequence of base-4 string indices (t_1 most significant)."""
    arr = (ctypes.c_ulonglong * max(len(strings), 1))(*[int(x) for x in strings])
    return int(load().tpd_partial_prepare(n, dtype, _opt(opt), arr, len(strings), workspace or None,
                                          workspace_bytes, stream or None))


def tpd_decompose_partial(A_ptr, n, dtype, opt, count, workspace, workspace_bytes, weights, stream=0):
    return int(load().tpd_decompose_partial(A_ptr or None, n, dtype, _opt(opt), count, workspace or None,
                                            workspace_bytes, weights or None, stream or None))


def tpd_sparse_workspace_size(max_entries):
    return int(load().tpd_sparse_workspace_size(max_entries))


def tpd_decompose_coo(rows, cols, values, nnz, n, dtype, max_entries, strings, weights, capacity, count, status,
                      workspace, workspace_bytes, stream=0):
    return int(load().tpd_decompose_coo(rows or None, cols or None, values or None, nnz, n, dtype, max_entries,
                                        strings or None, weights or None, capacity, count or None, status or None,
                                        workspace or None, workspace_bytes, stream or None))


def tpd_nonzero_workspace_size(n):
    return int(load().tpd_nonzero_workspace_size(n))


def tpd_nonzero_list(W, n, dtype, tol, strings, weights, capacity, count, workspace, workspace_bytes, stream=0):
    return int(load().tpd_nonzero_list(W or None, n, dtype, float(tol), strings or None, weights or None, capacity,
                                       count or None, workspace or None, workspace_bytes, stream or None))


def tpd_weyl_decompose(A, n, d, dtype, opt=None, stream=0):
    return int(load().tpd_weyl_decompose(A or None, n, d, dtype, _opt(opt), stream or None))


def tpd_weyl_compose(C, n, d, dtype, scale, opt=None, stream=0):
    return int(load().tpd_weyl_compose(C or None, n, d, dtype, float(scale), _opt(opt), stream or None))


def tpd_gellmann_decompose(A, n, d, dtype, opt=None, stream=0):
    return int(load().tpd_gellmann_decompose(A or None, n, d, dtype, _opt(opt), stream or None))


def tpd_gellmann_compose(C, n, d, dtype, scale, opt=None, stream=0):
    return int(load().tpd_gellmann_compose(C or None, n, d, dtype, float(scale), _opt(opt), stream or None))


def tpd_convert_layout(src, dst, n, dtype, to_string, stream=0):
    return int(load().tpd_convert_layout(src or None, dst or None, n, dtype, int(to_string), stream or None))


def tpd_sum_squares(x, count, dtype, result, workspace, workspace_bytes, stream=0):
    return int(load().tpd_sum_squares(x or None, count, dtype, result or None, workspace or None, workspace_bytes,
                                      stream or None))


def tpd_batch_status(workspace, stream=0):
    return int(load().tpd_batch_status(workspace, stream or None))


def tpd_test_hold_batch_waits(on):
    load().tpd_test_hold_batch_waits(int(bool(on)))


def tpd_decompose_noalloc(A_ptr, n, dtype, opt=None, stream=0):
    """Decomposition with the library's own fixed scratch array (no allocation)."""
    return int(load().tpd_decompose_noalloc(A_ptr, n, dtype, _opt(opt), stream or None))


def tpd_decompose_host(A_host_ptr, W_host_ptr, dev_ptr, n, dtype, opt=None, workspace=0, workspace_bytes=0,
                       stream=0):
    return int(load().tpd_decompose_host(A_host_ptr, W_host_ptr, dev_ptr, n, dtype, _opt(opt), workspace or None,
                                         workspace_bytes, stream or None))


def _int_array(values):
    arr = (ctypes.c_int * len(values))(*[int(v) for v in values])
    return arr


def tpd_batched_workspace_size(ns, dtype, opt=None):
    arr = _int_array(ns)
    return int(load().tpd_batched_workspace_size(arr, len(ns), dtype, _opt(opt)))


def tpd_decompose_batched(ptrs_dev, ns_dev, ns, dtype, opt=None, workspace=0, workspace_bytes=0, stream=0):
    arr = _int_array(ns)
    return int(load().tpd_decompose_batched(ptrs_dev, ns_dev, arr, len(ns), dtype, _opt(opt),
                                            workspace or None, workspace_bytes, stream or None))


def tpd_compose_batched(ptrs_dev, ns_dev, ns, dtype, scale_mode, opt=None, workspace=0, workspace_bytes=0,
                        stream=0):
    arr = _int_array(ns)
    return int(load().tpd_compose_batched(ptrs_dev, ns_dev, arr, len(ns), dtype, int(scale_mode), _opt(opt),
                                          workspace or None, workspace_bytes, stream or None))


def tpd_plan_describe(n, dtype, opt=None):
    buf = ctypes.create_string_buffer(8192)
    npass = load().tpd_plan_describe(n, dtype, _opt(opt), buf, len(buf))
    return npass, buf.value.decode()


def tpd_version():
    return int(load().tpd_version())
