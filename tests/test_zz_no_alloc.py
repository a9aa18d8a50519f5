"""tpd_decompose_noalloc: the decomposition for callers that may not allocate
device memory (a custom allocator owns the GPU, or a path that must never
allocate or synchronise).  Its workspace is the library's own fixed device
array instead of a caller buffer.  Checked through the C ABI against
tpd_decompose with a caller-allocated workspace, on consecutive calls, so a
second call that inherits the first call's scratch contents must still be
right.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2310_13421_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_13421_gb300 import buildlib, _lib
    buildlib.build()
    _lib.load()
    return _lib


def _reference(L, A, n, opt):
    out = A.clone()
    wsb = L.tpd_workspace_size(n, L.TPD_C128, opt)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    st = L.tpd_decompose(out.data_ptr(), n, L.TPD_C128, opt, ws.data_ptr(), wsb,
                         torch.cuda.current_stream().cuda_stream)
    assert st == L.TPD_OK, L.status_string(st)
    return out


def _noalloc(L, A, n, opt):
    out = A.clone()
    st = L.tpd_decompose_noalloc(out.data_ptr(), n, L.TPD_C128, opt, torch.cuda.current_stream().cuda_stream)
    assert st == L.TPD_OK, L.status_string(st)
    return out


def test_noalloc_matches_decompose_on_consecutive_calls(L):
    # multi-pass plans hand their per-class binary points (and, with zero
    # skipping, per-tile flags) to one another in the scratch array
    cases = [
        (12, synth.hermitian(12, seed=31), L.options(skip_zero=True)),
        (12, synth.heisenberg(12, *synth.heisenberg_params(12, seed=32)), L.options(skip_zero=True)),
        (14, synth.hermitian(14, seed=33), L.options(skip_zero=True)),
        (12, synth.general(12, seed=34), L.options(skip_zero=True)),
        (12, synth.general(12, seed=35), L.options()),
    ]
    assert 0 < max(L.tpd_workspace_size(n, L.TPD_C128, opt) for n, _, opt in cases) <= L.TPD_NOALLOC_SCRATCH_BYTES
    for n, A, opt in cases:
        At = torch.from_numpy(A).cuda()
        want = _reference(L, At, n, opt)
        got1 = _noalloc(L, At, n, opt)
        got2 = _noalloc(L, At, n, opt)      # second call in a row reuses the array as left
        torch.cuda.synchronize()
        # the same plan and arithmetic: identical bits (a stale flag would show)
        assert torch.equal(got1, want)
        assert torch.equal(got2, want)


def test_noalloc_rejects_plans_larger_than_its_array(L):
    # 2^9-element tiles at n = 16 need gigabytes of binary points: refused
    # before any launch
    opt = L.options(tile_bits=9, skip_zero=True)
    assert L.tpd_workspace_size(16, L.TPD_C128, opt) > L.TPD_NOALLOC_SCRATCH_BYTES
    A = torch.zeros(16, dtype=torch.complex128, device="cuda")   # never touched
    st = L.tpd_decompose_noalloc(A.data_ptr(), 16, L.TPD_C128, opt, torch.cuda.current_stream().cuda_stream)
    assert st == L.TPD_ERR_WORKSPACE
