"""GPU: the torch front end on a caller's side stream.  Work enqueued on a
stream other than the current one must run after what the current stream has
already enqueued (which produced its input), and tensors it allocates or
reads must not be handed to other work by the caching allocator while that
stream still uses them."""
import numpy as np
import pytest

from paper_2310_13421_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def test_side_stream_waits_for_its_input(tpd):
    n = 12
    src = torch.from_numpy(synth.hermitian(n, seed=9900)).cuda()
    want = tpd.decompose(src, skip_zero=True)
    want_back = tpd.compose(want, scale=2.0 ** -n)
    want_str = tpd.to_string_layout(want)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    for _ in range(3):
        X = torch.empty_like(src)
        torch.cuda._sleep(2_000_000)        # keep the current stream busy ...
        X.copy_(src)                        # ... so the input is written late
        got = tpd.decompose(X, skip_zero=True, stream=side)
        Y = X.clone()
        tpd.decompose(Y, inplace=True, stream=side)
        del X                               # freed while the side stream may still read it
        junk = torch.full_like(src, 7.0)    # would reuse X's memory if it were not recorded on side
        back = tpd.compose(got, scale=2.0 ** -n, stream=side)
        s = tpd.to_string_layout(got, stream=side)
        side.synchronize()
        torch.cuda.synchronize()
        assert torch.equal(got, want)
        assert torch.equal(Y, want)
        assert torch.equal(back, want_back)
        assert torch.equal(s, want_str)
        del junk
