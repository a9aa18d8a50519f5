"""GPU at the largest size: n = 16 (a 65536 x 65536 matrix; 64 GB in
complex128, 32 GB in complex64).  The oracle cannot run at this size, so the
checks are what holds at any size: the planted Heisenberg chain's weights
(closed form, pinned against the oracle at small n) exactly, and Parseval's
identity for a random matrix."""
import numpy as np
import pytest

from paper_2310_13421_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if torch.cuda.get_device_properties(0).total_memory < 100 * 2 ** 30:
        pytest.skip("needs a GPU with more than 100 GB")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def test_n16_planted_heisenberg_complex128(tpd):
    n = 16
    J, h = synth.heisenberg_params(n, seed=9960)
    H = torch.zeros((1 << n, 1 << n), dtype=torch.complex128, device="cuda")
    synth.heisenberg_into(H, n, J, h)
    tpd.decompose(H, inplace=True)
    s, w = tpd.nonzero_list(H)
    want = sorted((synth.string_index(t), v) for t, v in synth.heisenberg_terms(n, J, h).items())
    assert s.cpu().tolist() == [k for k, _ in want]
    assert np.array_equal(w.cpu().numpy(), np.array([v for _, v in want], dtype=np.complex128))
    del H
    torch.cuda.empty_cache()


def test_n16_parseval_complex64(tpd):
    n = 16
    g = torch.Generator(device="cuda").manual_seed(9961)
    A = torch.randn((1 << n, 1 << n), dtype=torch.complex64, device="cuda", generator=g)
    a2 = float(tpd.sum_squares(A))
    for prec in ("compensated", "plain"):
        W = tpd.decompose(A, precision=prec)
        w2 = float(tpd.sum_squares(W))
        # each pass is 2^-1/2-scaled unitary per level: ||A||^2 = 2^n sum |w|^2 up to the rounding
        assert abs(w2 * 2 ** n - a2) <= 8 * n * 2.0 ** -24 * a2, prec
        del W
        torch.cuda.empty_cache()
