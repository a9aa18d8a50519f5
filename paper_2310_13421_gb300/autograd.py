"""torch.autograd.Function for the Pauli decomposition.

The decomposition D is linear with adjoint D^H = 2^-n C, C the composition:
the Pauli strings are Hermitian (Sec. II.A), so the matrix of D has rows
2^-n conj(sigma^t) and its conjugate transpose has columns 2^-n sigma^t.  For
a complex linear map torch's backward applies the adjoint to the incoming
gradient, so backward(g) = 2^-n C(g), run by the composition kernel.
"""
import torch

from . import api


class TPDFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, precision=None):
        ctx.precision = precision
        return api.decompose(A, inplace=False, precision=precision)

    @staticmethod
    def backward(ctx, g):
        n = int(g.shape[0]).bit_length() - 1
        gin = api.compose(g.contiguous(), scale=2.0 ** -n, inplace=False, precision=ctx.precision)
        return gin, None


def tpd(A, precision=None):
    """Differentiable decomposition: weights of A in RC layout."""
    return TPDFunction.apply(A, precision)
