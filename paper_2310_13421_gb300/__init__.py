"""GB300-native tensorized Pauli decomposition (arXiv:2310.13421).

The CUDA library ``libtpd.so`` is loaded lazily on first use (the submodule
``synth`` imports without a GPU or torch).  Public API:

    decompose(A, ...)          Pauli weights of a 2^n x 2^n CUDA matrix (in place or copy)
    compose(C, scale=...)      scale * sum_t w_t sigma^t (the adjoint for scale 2^-n)
    decompose_batched(mats)    many matrices of different sizes in one call
    Batch                      reusable device batch descriptor (CUDA-graph friendly)
    TPDFunction / tpd          autograd
    string_order(n)            RC layout -> string order permutation
    build()                    compile libtpd.so in-tree
"""
__all__ = ["decompose", "compose", "decompose_batched", "compose_batched", "Batch", "TPDFunction", "tpd",
           "string_order", "workspace_size", "build"]


def build(force=False, verbose=False):
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)


def __getattr__(name):
    if name in ("decompose", "compose", "decompose_batched", "compose_batched", "Batch", "string_order",
                "workspace_size", "make_options"):
        from . import api
        return getattr(api, name)
    if name in ("TPDFunction", "tpd"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
