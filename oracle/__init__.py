"""Plain CPU oracle for the Pauli decomposition of arXiv:2310.13421.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path (``paper_2310_13421_gb300``) and never imports it.

Two independent evaluations of Eq. 2, w_t = 2^-n tr(sigma^t A):

* ``kron``  -- O0: explicit Kronecker products (Eq. 1) and a dense trace, numpy,
  n <= 4.  Used to pin the C oracle.
* ``core``  -- O1/O2: the trace written out over the one nonzero per row of a
  Pauli string (C, OpenMP, fp64); see ``tpd_oracle.c``.

and the paper's own algorithm on the CPU (``tpd_alg2``: the iterative Alg. 2,
the CMWs of Eq. 4 level by level in place, OpenMP, in ``tpd_alg2.c``): the
algorithmic CPU baseline, pinned in the tests against the two evaluations
above.

Coefficient layout everywhere in the oracle: STRING order, index
s = sum_j t_j 4^(n-j) with t_1 (the first tensor factor) most significant and
t in {0,1,2,3} = {I,X,Y,Z}.
"""
from .core import (coeffs, coeffs_at, coeffs_fwht, coeffs_xrows, compose, compose_fwht, grad_weighted_sq,
                   num_threads, string_of_xz, build_library, tpd_alg2)
from .kron import pauli_string_matrix, coeffs_kron, compose_kron

__all__ = [
    "coeffs", "coeffs_at", "coeffs_fwht", "coeffs_xrows", "compose", "compose_fwht", "grad_weighted_sq",
    "num_threads", "string_of_xz", "build_library", "tpd_alg2",
    "pauli_string_matrix", "coeffs_kron", "compose_kron",
]
