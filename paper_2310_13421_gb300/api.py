"""Torch-level front end: marshals tensors, streams and workspaces to the C ABI
(_lib).  Every step of the decomposition runs in libtpd.so's kernels; there is
no other code path.

Layout reminder: results are IN the input's storage order ("RC layout"): the
weight of string t sits at row r, column c with, for every qubit j, the row
and column bits n-j equal to (t_j >> 1, t_j & 1) -- I (0,0), X (0,1), Y (1,0),
Z (1,1).  ``to_string_layout`` converts to base-4 string order on the device.
"""
import contextlib

import numpy as np
import torch

from . import _lib as L

_PREC = {
    "default": L.TPD_PREC_DEFAULT, None: L.TPD_PREC_DEFAULT,
    "plain": L.TPD_PREC_PLAIN, "fp64": L.TPD_PREC_PLAIN, "fp32": L.TPD_PREC_PLAIN,
    "compensated": L.TPD_PREC_COMPENSATED,
    "fixed": L.TPD_PREC_FIXED,
}


def _dtype_code(t):
    if t.dtype == torch.complex128:
        return L.TPD_C128
    if t.dtype == torch.complex64:
        return L.TPD_C64
    raise TypeError("expected complex128 or complex64, got %s" % t.dtype)


def _qubits(t):
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("expected a square matrix, got shape %s" % (tuple(t.shape),))
    N = int(t.shape[0])
    if N < 2 or N & (N - 1):
        raise ValueError("matrix side must be a power of two >= 2, got %d" % N)
    return N.bit_length() - 1


def _check_device(t):
    if not t.is_cuda:
        raise ValueError("tensor must be on a CUDA device (the decomposition runs only in libtpd.so)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous (row-major)")


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@contextlib.contextmanager
def _enqueue(device, stream, *inputs):
    """Device and stream (yields the cudaStream_t) for enqueueing library
    work.  The work and every tensor made for it inside the block (a clone of
    the input, a workspace, the outputs) belong to `stream` (default: the
    current stream).  A stream other than the current one first waits for
    the work already enqueued on the current stream, which produced the
    inputs, and the inputs are recorded on it, so that the caching allocator
    does not hand their memory to other work while the stream still uses
    them.  Results are ready on `stream`."""
    with torch.cuda.device(device):
        cur = torch.cuda.current_stream()
        s = stream if stream is not None else cur
        if s != cur:
            s.wait_stream(cur)
            for t in inputs:
                if t is not None:
                    t.record_stream(s)
        with torch.cuda.stream(s):
            yield s.cuda_stream


def _raise(st, what):
    if st != L.TPD_OK:
        raise L.TPDError(st, what)


def make_options(precision=None, skip_zero=False, tile_bits=0, max_levels=0, variant=0, l2_chunk_mb=0):
    if isinstance(precision, str) or precision is None:
        precision = _PREC[precision]
    return L.options(precision, skip_zero, tile_bits, max_levels, variant, l2_chunk_mb=l2_chunk_mb)


def workspace_size(n, dtype, **kw):
    code = L.TPD_C128 if dtype in (torch.complex128, L.TPD_C128) else L.TPD_C64
    return L.tpd_workspace_size(n, code, make_options(**kw))


def decompose(A, *, inplace=False, precision=None, skip_zero=False, tile_bits=0, max_levels=0, variant=0,
              l2_chunk_mb=0, workspace=None, stream=None):
    """Pauli weights w_t = 2^-n tr(sigma^t A) of a 2^n x 2^n CUDA matrix, in RC layout."""
    _check_device(A)
    n = _qubits(A)
    code = _dtype_code(A)
    opt = make_options(precision, skip_zero, tile_bits, max_levels, variant, l2_chunk_mb)
    wsb = L.tpd_workspace_size(n, code, opt)
    with _enqueue(A.device, stream, A, workspace) as s:
        out = A if inplace else A.clone()
        ws = workspace
        if wsb and (ws is None or ws.numel() < wsb):
            ws = torch.empty(wsb, dtype=torch.uint8, device=A.device)
        st = L.tpd_decompose(out.data_ptr(), n, code, opt, ws.data_ptr() if wsb else 0, wsb, s)
    _raise(st, "tpd_decompose")
    return out


def compose(C, *, scale=1.0, inplace=False, precision=None, skip_zero=False, tile_bits=0, max_levels=0, variant=0,
            workspace=None, stream=None):
    """scale * sum_t w_t sigma^t from weights in RC layout (scale 2^-n: the adjoint of decompose)."""
    _check_device(C)
    n = _qubits(C)
    code = _dtype_code(C)
    opt = make_options(precision, skip_zero, tile_bits, max_levels, variant)
    wsb = L.tpd_workspace_size(n, code, opt)
    with _enqueue(C.device, stream, C, workspace) as s:
        out = C if inplace else C.clone()
        ws = workspace
        if wsb and (ws is None or ws.numel() < wsb):
            ws = torch.empty(wsb, dtype=torch.uint8, device=C.device)
        st = L.tpd_compose(out.data_ptr(), n, code, float(scale), opt, ws.data_ptr() if wsb else 0, wsb, s)
    _raise(st, "tpd_compose")
    return out


class Batch:
    """Device-side descriptor of a list of matrices for the batched calls
    (pointer and qubit arrays plus workspace), reusable across calls and
    CUDA-graph captures as long as the matrices stay in place."""

    def __init__(self, mats, precision=None, tile_bits=0, max_levels=0, variant=0):
        if not mats:
            raise ValueError("empty batch")
        dev = mats[0].device
        self.code = _dtype_code(mats[0])
        self.ns = []
        for m in mats:
            _check_device(m)
            if _dtype_code(m) != self.code or m.device != dev:
                raise ValueError("batch matrices must share dtype and device")
            self.ns.append(_qubits(m))
        self.mats = list(mats)
        self.opt = make_options(precision, False, tile_bits, max_levels, variant)
        self.ptrs = torch.tensor([m.data_ptr() for m in mats], dtype=torch.int64, device=dev)
        self.ns_dev = torch.tensor(self.ns, dtype=torch.int32, device=dev)
        wsb = L.tpd_batched_workspace_size(self.ns, self.code, self.opt)
        if wsb == 0:
            raise ValueError("invalid batch (qubit counts must be 1..12)")
        self.ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        self.device = dev

    def _inputs(self):
        return [self.ptrs, self.ns_dev, self.ws] + self.mats

    def decompose(self, stream=None):
        with _enqueue(self.device, stream, *self._inputs()) as s:
            st = L.tpd_decompose_batched(self.ptrs.data_ptr(), self.ns_dev.data_ptr(), self.ns, self.code,
                                         self.opt, self.ws.data_ptr(), self.ws.numel(), s)
        _raise(st, "tpd_decompose_batched")

    def status(self, stream=None):
        """Status word of the last call (waits for the stream): 0 = OK; see tpd_batch_status."""
        with torch.cuda.device(self.device):
            return L.tpd_batch_status(self.ws.data_ptr(), _stream(stream))

    def compose(self, adjoint=False, stream=None):
        with _enqueue(self.device, stream, *self._inputs()) as s:
            st = L.tpd_compose_batched(self.ptrs.data_ptr(), self.ns_dev.data_ptr(), self.ns, self.code,
                                       1 if adjoint else 0, self.opt, self.ws.data_ptr(), self.ws.numel(), s)
        _raise(st, "tpd_compose_batched")


def decompose_batched(mats, *, inplace=False, precision=None, variant=0, stream=None):
    """Decompose a list of CUDA matrices of (possibly different) sizes; one
    call enqueues the whole batch (one launch per qubit count and pass; with
    variant=2 a single persistent kernel launch)."""
    work = list(mats) if inplace else [m.clone() for m in mats]
    Batch(work, precision=precision, variant=variant).decompose(stream)
    return work


def compose_batched(mats, *, adjoint=False, inplace=False, precision=None, variant=0, stream=None):
    work = list(mats) if inplace else [m.clone() for m in mats]
    Batch(work, precision=precision, variant=variant).compose(adjoint=adjoint, stream=stream)
    return work


class Partial:
    """Partial decomposition (Alg. 3): the weights of a fixed list of strings
    (base-4 indices, t_1 most significant) for matrices of one size and dtype.
    The host-side preparation runs once; ``decompose`` can then be called (and
    captured in a CUDA graph) repeatedly."""

    def __init__(self, n, strings, dtype=torch.complex128, device="cuda", precision=None, tile_bits=0,
                 max_levels=0):
        self.n = int(n)
        self.code = L.TPD_C128 if dtype == torch.complex128 else L.TPD_C64
        self.dtype = dtype
        self.count = len(strings)
        self.opt = make_options(precision, False, tile_bits, max_levels)
        wsb = L.tpd_partial_workspace_size(self.n, self.code, self.opt, self.count)
        if wsb == 0:
            raise ValueError("invalid partial decomposition arguments")
        self.ws = torch.empty(wsb, dtype=torch.uint8, device=device)
        self.device = self.ws.device
        with torch.cuda.device(self.device):
            st = L.tpd_partial_prepare(self.n, self.code, self.opt, list(strings), self.ws.data_ptr(), wsb,
                                       _stream(None))
        _raise(st, "tpd_partial_prepare")

    def decompose(self, A, *, inplace=False, out=None, stream=None):
        """Requested weights (a 1-D tensor in request order); A is consumed
        when inplace (its other elements are then unspecified)."""
        _check_device(A)
        if _qubits(A) != self.n or _dtype_code(A) != self.code:
            raise ValueError("matrix does not match the prepared size / dtype")
        with _enqueue(A.device, stream, A, self.ws, out) as s:
            work = A if inplace else A.clone()
            if out is None:
                out = torch.empty(self.count, dtype=self.dtype, device=A.device)
            st = L.tpd_decompose_partial(work.data_ptr(), self.n, self.code, self.opt, self.count, self.ws.data_ptr(),
                                         self.ws.numel(), out.data_ptr(), s)
        _raise(st, "tpd_decompose_partial")
        return out


def decompose_coo(rows, cols, values, n, *, max_entries=None, capacity=None, stream=None):
    """Pauli weights of a sparse complex128 2^n x 2^n matrix given by its
    nonzero entries (CUDA tensors rows, cols: int32, values: complex128):
    the paper's list L as (string indices, weights), sorted by string index.
    max_entries: entries a level may hold (default 4 * nnz + 1024, doubled
    and retried while too small); synchronises to read the count."""
    for t in (rows, cols, values):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("rows, cols, values must be contiguous CUDA tensors")
    if rows.dtype != torch.int32 or cols.dtype != torch.int32 or values.dtype != torch.complex128:
        raise TypeError("rows, cols: int32; values: complex128")
    nnz = values.numel()
    dev = values.device
    cap_entries = int(max_entries) if max_entries else 4 * nnz + 1024
    while True:
        with _enqueue(dev, stream, rows, cols, values) as s:
            count = torch.zeros(1, dtype=torch.int64, device=dev)
            status = torch.zeros(1, dtype=torch.int32, device=dev)
            ws = torch.empty(L.tpd_sparse_workspace_size(cap_entries), dtype=torch.uint8, device=dev)
            cap = int(capacity) if capacity is not None else cap_entries
            strings = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
            weights = torch.empty(max(cap, 1), dtype=torch.complex128, device=dev)
            st = L.tpd_decompose_coo(rows.data_ptr(), cols.data_ptr(), values.data_ptr(), nnz, int(n), L.TPD_C128,
                                     cap_entries, strings.data_ptr(), weights.data_ptr(), cap, count.data_ptr(),
                                     status.data_ptr(), ws.data_ptr(), ws.numel(), s)
        _raise(st, "tpd_decompose_coo")
        if int(status.item()) == 0:
            k = min(int(count.item()), cap)
            return strings[:k], weights[:k]
        if max_entries:
            raise L.TPDError(L.TPD_ERR_WORKSPACE, "tpd_decompose_coo (max_entries too small)")
        cap_entries *= 2


def nonzero_list(W, *, tol=0.0, capacity=None, stream=None):
    """The paper's list L: (string indices, weights) of the weights in W (RC
    layout) with |re| > tol or |im| > tol, in increasing string index.
    Synchronises to size the result unless `capacity` is given."""
    _check_device(W)
    n = _qubits(W)
    code = _dtype_code(W)
    with _enqueue(W.device, stream, W) as s:
        ws = torch.empty(L.tpd_nonzero_workspace_size(n), dtype=torch.uint8, device=W.device)
        count = torch.zeros(1, dtype=torch.int64, device=W.device)
        if capacity is None:
            st = L.tpd_nonzero_list(W.data_ptr(), n, code, tol, 0, 0, 0, count.data_ptr(), ws.data_ptr(),
                                    ws.numel(), s)
            _raise(st, "tpd_nonzero_list")
            cap = int(count.item())
        else:
            cap = int(capacity)
        strings = torch.empty(max(cap, 1), dtype=torch.int64, device=W.device)
        weights = torch.empty(max(cap, 1), dtype=W.dtype, device=W.device)
        st = L.tpd_nonzero_list(W.data_ptr(), n, code, tol, strings.data_ptr(), weights.data_ptr(), cap,
                                count.data_ptr(), ws.data_ptr(), ws.numel(), s)
    _raise(st, "tpd_nonzero_list")
    if capacity is None:
        return strings[:cap], weights[:cap]
    return strings, weights, count


def to_string_layout(W, *, stream=None):
    """Weights in STRING layout (base-4 string index, t_1 most significant) as
    a flat tensor, converted from the RC layout on the device."""
    _check_device(W)
    n = _qubits(W)
    with _enqueue(W.device, stream, W) as s:
        out = torch.empty(W.numel(), dtype=W.dtype, device=W.device)
        st = L.tpd_convert_layout(W.data_ptr(), out.data_ptr(), n, _dtype_code(W), 1, s)
    _raise(st, "tpd_convert_layout")
    return out


def from_string_layout(S, *, stream=None):
    """Inverse of to_string_layout: a flat STRING-layout tensor of 4^n weights
    back to the N x N RC layout."""
    if not S.is_cuda or not S.is_contiguous():
        raise ValueError("tensor must be a contiguous CUDA tensor")
    m = S.numel()
    n = (m.bit_length() - 1) // 2
    if m < 4 or 4 ** n != m:
        raise ValueError("expected 4^n elements, got %d" % m)
    with _enqueue(S.device, stream, S) as s:
        out = torch.empty((2 ** n, 2 ** n), dtype=S.dtype, device=S.device)
        st = L.tpd_convert_layout(S.data_ptr(), out.data_ptr(), n, _dtype_code(S), 0, s)
    _raise(st, "tpd_convert_layout")
    return out


def sum_squares(X, *, stream=None):
    """sum |x|^2 over a complex CUDA tensor, in fp64 on the device (a 0-dim
    float64 CUDA tensor; deterministic)."""
    _check_device(X)
    with _enqueue(X.device, stream, X) as s:
        out = torch.empty((), dtype=torch.float64, device=X.device)
        ws = torch.empty(L.TPD_SUMSQ_WORKSPACE_BYTES, dtype=torch.uint8, device=X.device)
        st = L.tpd_sum_squares(X.data_ptr(), X.numel(), _dtype_code(X), out.data_ptr(), ws.data_ptr(), ws.numel(), s)
    _raise(st, "tpd_sum_squares")
    return out


def _qudits(t, d):
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError("expected a square matrix, got shape %s" % (tuple(t.shape),))
    N, n = int(t.shape[0]), 0
    while d ** n < N:
        n += 1
    if n < 1 or d ** n != N:
        raise ValueError("matrix side must be a power of d = %d, got %d" % (d, N))
    return n


def weyl_decompose(A, d, *, inplace=False, precision=None, stream=None):
    """Weights c_{a,b} = d^-n tr(W_{a,b}^* A) of a d^n x d^n CUDA matrix in the
    Weyl (clock-and-shift) basis W_{a,b} = X^a Z^b; the weight of (a, b)
    sits at row digits b, column digits a + b mod d (see tpd_weyl_decompose).
    precision: None / "fixed" (complex128, d <= 4: block fixed point) or
    "plain" (IEEE, rounded every level)."""
    _check_device(A)
    n = _qudits(A, d)
    opt = make_options(precision)
    with _enqueue(A.device, stream, A) as s:
        out = A if inplace else A.clone()
        st = L.tpd_weyl_decompose(out.data_ptr(), n, int(d), _dtype_code(A), opt, s)
    _raise(st, "tpd_weyl_decompose")
    return out


def weyl_compose(C, d, *, scale=1.0, inplace=False, precision=None, stream=None):
    """scale * sum c_{a,b} W_{a,b} from weights in the layout of weyl_decompose
    (scale d^-n: its adjoint); precision as for weyl_decompose."""
    _check_device(C)
    n = _qudits(C, d)
    opt = make_options(precision)
    with _enqueue(C.device, stream, C) as s:
        out = C if inplace else C.clone()
        st = L.tpd_weyl_compose(out.data_ptr(), n, int(d), _dtype_code(C), float(scale), opt, s)
    _raise(st, "tpd_weyl_compose")
    return out


def gellmann_decompose(A, d, *, inplace=False, precision=None, stream=None):
    """Coefficients g_(r,c) = tr(G_(r,c) A) / tr(G_(r,c)^2) of a d^n x d^n CUDA
    matrix in the generalized Gell-Mann basis (identity, diagonal,
    symmetric and antisymmetric elements; d = 2: the Pauli basis); g_(r,c)
    sits at row r, column c (see tpd_gellmann_decompose).  IEEE arithmetic
    of the storage type; precision None or "plain"."""
    _check_device(A)
    n = _qudits(A, d)
    opt = make_options(precision)
    with _enqueue(A.device, stream, A) as s:
        out = A if inplace else A.clone()
        st = L.tpd_gellmann_decompose(out.data_ptr(), n, int(d), _dtype_code(A), opt, s)
    _raise(st, "tpd_gellmann_decompose")
    return out


def gellmann_compose(C, d, *, scale=1.0, inplace=False, precision=None, stream=None):
    """scale * sum g_(r,c) G_(r,c) from coefficients in the layout of
    gellmann_decompose (scale 1: its inverse)."""
    _check_device(C)
    n = _qudits(C, d)
    opt = make_options(precision)
    with _enqueue(C.device, stream, C) as s:
        out = C if inplace else C.clone()
        st = L.tpd_gellmann_compose(out.data_ptr(), n, int(d), _dtype_code(C), float(scale), opt, s)
    _raise(st, "tpd_gellmann_compose")
    return out


def string_order(n):
    """Index array p with p[s] = flat RC position of string s (base-4 string
    index, t_1 most significant): rc_tensor.flatten()[p] is in string order."""
    s = np.arange(4 ** n, dtype=np.int64)
    r = np.zeros_like(s)
    c = np.zeros_like(s)
    for beta in range(n):
        t = (s >> (2 * beta)) & 3
        r |= (t >> 1) << beta
        c |= (t & 1) << beta
    return r * (1 << n) + c
