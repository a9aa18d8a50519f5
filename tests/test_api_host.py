"""CPU: the torch-facing API has no CPU fallback -- a host tensor is refused
with an error naming the CUDA library before anything is computed -- and the
qudit-basis calls check the matrix side against d before any launch."""
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_2310_13421_gb300 import api as a
    return a


@pytest.mark.parametrize("fn,args", [
    ("decompose", ()), ("compose", ()), ("weyl_decompose", (3,)), ("weyl_compose", (3,)),
    ("gellmann_decompose", (3,)), ("gellmann_compose", (3,)),
])
def test_host_tensors_are_refused(api, fn, args):
    side = 9 if args else 8
    A = torch.zeros(side, side, dtype=torch.complex128)
    with pytest.raises(ValueError, match="CUDA"):
        getattr(api, fn)(A, *args)


def test_qudit_side_must_be_a_power_of_d(api):
    for bad in (torch.zeros(8, 8, dtype=torch.complex128), torch.zeros(9, 3, dtype=torch.complex128)):
        with pytest.raises(ValueError):
            api._qudits(bad, 3)
    assert api._qudits(torch.zeros(27, 27, dtype=torch.complex128), 3) == 3
    assert api._qudits(torch.zeros(25, 25, dtype=torch.complex64), 5) == 2
