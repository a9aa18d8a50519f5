"""GB300-native tensorized Pauli decomposition (arXiv:2310.13421).

The CUDA library ``libtpd.so`` is loaded lazily on first use (the submodule
``synth`` imports without a GPU or torch).  Public API:

    decompose(A, ...)          Pauli weights of a 2^n x 2^n CUDA matrix (in place or copy)
    compose(C, scale=...)      scale * sum_t w_t sigma^t (the adjoint for scale 2^-n)
    decompose_batched(mats)    many matrices of different sizes in one call
    Batch                      reusable device batch descriptor (CUDA-graph friendly)
    Partial                    partial decomposition: weights of a list of strings only (Alg. 3)
    TPDFunction / tpd          autograd
    to_string_layout(W)        RC -> base-4 string order (device kernel); from_string_layout inverse
    sum_squares(X)             fp64 sum of |x|^2 on the device (Parseval check)
    nonzero_list(W)            the paper's list L of (string, weight) with nonzero weight
    decompose_coo(r, c, v, n)  sparse input: the list L from the nonzero entries (Alg. 2 on entries)
    weyl_decompose(A, d)       the same recursion in the Weyl (clock-and-shift) basis of qudits (Sec. V)
    weyl_compose(C, d)         its inverse / adjoint
    gellmann_decompose(A, d)   the same recursion in the generalized Gell-Mann basis of qudits (Sec. V)
    gellmann_compose(C, d)     its inverse
    string_order(n)            RC layout -> string order permutation (host index array)
    build()                    compile libtpd.so in-tree
"""
__all__ = ["decompose", "compose", "decompose_batched", "compose_batched", "Batch", "Partial", "TPDFunction", "tpd",
           "string_order", "to_string_layout", "from_string_layout", "sum_squares", "nonzero_list", "decompose_coo",
           "workspace_size", "weyl_decompose", "weyl_compose", "gellmann_decompose", "gellmann_compose",
           "build"]


def build(force=False, verbose=False):
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("decompose", "compose", "decompose_batched", "compose_batched", "Batch", "Partial", "string_order",
                "to_string_layout", "from_string_layout", "sum_squares", "nonzero_list", "decompose_coo",
                "workspace_size", "make_options", "weyl_decompose", "weyl_compose", "gellmann_decompose",
                "gellmann_compose"):
        from . import api
        return getattr(api, name)
    if name in ("TPDFunction", "tpd"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
