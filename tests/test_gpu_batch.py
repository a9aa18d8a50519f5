"""GPU: the batched calls in their two forms -- one launch per (qubit count,
pass) (default) and one persistent kernel launch (variant 2) -- against the CPU oracle and
against each other, CUDA-graph replay of the persistent form, and its status
word: a bounded wait that runs out (test hook) and device qubit counts that
disagree with the host's, both reported without a fault."""
import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import U32, assert_close, assert_exact, rel_err, to_string_order

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL128 = 1e-12
STATUS_OK, STATUS_INVALID, STATUS_TIMEOUT = 0, 1, 6


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def gpu(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def npass(n, dtype=0, prec=0):
    from paper_2310_13421_gb300 import _lib as L
    return L.tpd_plan_describe(n, dtype, L.options(precision=prec))[0]


def mixed_sizes(seed, count=40, lo=1, hi=10):
    rng = np.random.default_rng(seed)
    return [int(x) for x in list(range(lo, hi + 1)) + list(rng.integers(lo, hi + 1, size=count - (hi - lo + 1)))]


@pytest.mark.parametrize("precision", ["fixed", "plain"])
def test_persistent_matches_oracle_and_per_pass_form(tpd, precision):
    ns = mixed_sizes(9500)
    mats = [synth.general(n, seed=9500 + i) for i, n in enumerate(ns)]
    one = tpd.decompose_batched([gpu(m) for m in mats], precision=precision, variant=2)  # one launch
    per = tpd.decompose_batched([gpu(m) for m in mats], precision=precision)             # per (n, pass)
    for m, o, p, n in zip(mats, one, per, ns):
        want = oracle.coeffs_fwht(m)
        assert_close(to_string_order(host(o), n), want, TOL128, "persistent n=%d" % n)
        if precision == "fixed":
            # the same exact sums and one rounding: identical bits
            assert_exact(host(o), host(p), "persistent vs per-pass n=%d" % n)
        else:
            assert_close(to_string_order(host(p), n), want, TOL128, "per-pass n=%d" % n)


def test_persistent_integer_bit_exact_and_roundtrip(tpd):
    ns = mixed_sizes(9600)
    ints = [synth.int_general(n, seed=9600 + i) for i, n in enumerate(ns)]
    work = [gpu(m) for m in ints]
    batch = tpd.Batch(work, variant=2)
    batch.decompose()
    assert batch.status() == STATUS_OK
    for m, w, n in zip(ints, work, ns):
        assert_exact(to_string_order(host(w), n), oracle.coeffs_fwht(m), "n=%d" % n)
    batch.compose()                   # composition (Eq. 2) of the weights: A exactly
    assert batch.status() == STATUS_OK
    for m, w in zip(ints, work):
        assert_exact(host(w), m)
    batch.decompose()
    batch.compose(adjoint=True)       # the adjoint 2^-n C: 2^-n A, exact (power of two)
    for m, w, n in zip(ints, work, ns):
        assert_exact(host(w), m * 2.0 ** -n)


@pytest.mark.parametrize("precision", ["plain", "compensated"])
def test_persistent_c64(tpd, precision):
    ns = mixed_sizes(9700, count=24)
    mats = [synth.hermitian(n, seed=9700 + i, dtype=np.complex64) for i, n in enumerate(ns)]
    outs = tpd.decompose_batched([gpu(m, torch.complex64) for m in mats], precision=precision, variant=2)
    prec = 1 if precision == "plain" else 2
    for m, o, n in zip(mats, outs, ns):
        want = oracle.coeffs_fwht(m.astype(np.complex128))
        bound = n * U32 / (1 - n * U32) if precision == "plain" else (max(npass(n, 1, prec), 1) + 1) * U32
        assert rel_err(to_string_order(host(o), n), want) <= bound * 1.01, "c64 %s n=%d" % (precision, n)


def test_persistent_graph_replay(tpd):
    ns = [3, 5, 6, 7, 8, 10, 7, 4]
    mats = [synth.general(n, seed=9800 + i) for i, n in enumerate(ns)]
    work = [gpu(m) for m in mats]
    pristine = [w.clone() for w in work]
    batch = tpd.Batch(work, variant=2)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.decompose(stream=s)          # warm-up (plans, attributes) outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.decompose()
    for _ in range(3):
        for w, p in zip(work, pristine):
            w.copy_(p)
        g.replay()
        torch.cuda.synchronize()
        assert batch.status() == STATUS_OK
        for m, w, n in zip(mats, work, ns):
            assert_close(to_string_order(host(w), n), oracle.coeffs_fwht(m), TOL128, "graph n=%d" % n)


def test_bounded_wait_reports_timeout_and_context_survives(tpd):
    from paper_2310_13421_gb300 import _lib as L
    ns = [7, 8, 3, 9]                      # two-pass plans: their second passes wait
    mats = [synth.general(n, seed=9900 + i) for i, n in enumerate(ns)]
    work = [gpu(m) for m in mats]
    batch = tpd.Batch(work, variant=2)
    L.tpd_test_hold_batch_waits(1)
    try:
        batch.decompose()
        assert batch.status() == STATUS_TIMEOUT
    finally:
        L.tpd_test_hold_batch_waits(0)
    # the context is intact: a fresh call on new copies is correct and reports OK
    work2 = [gpu(m) for m in mats]
    batch2 = tpd.Batch(work2, variant=2)
    batch2.decompose()
    assert batch2.status() == STATUS_OK
    for m, w, n in zip(mats, work2, ns):
        assert_close(to_string_order(host(w), n), oracle.coeffs_fwht(m), TOL128, "after timeout n=%d" % n)


@pytest.mark.parametrize("variant", [0, 2])
def test_inconsistent_device_sizes_touch_nothing(tpd, variant):
    from paper_2310_13421_gb300 import _lib as L
    ns = [3, 7, 5, 8]
    mats = [synth.general(n, seed=9950 + i) for i, n in enumerate(ns)]
    work = [gpu(m) for m in mats]
    batch = tpd.Batch(work, variant=variant)
    # the device copy of the qubit counts disagrees with the host's
    batch.ns_dev.copy_(torch.tensor([3, 7, 5, 7], dtype=torch.int32, device="cuda"))
    batch.decompose()
    assert batch.status() == STATUS_INVALID
    for m, w in zip(mats, work):
        assert_exact(host(w), m)
    assert L.TPD_ERR_INVALID_ARG == STATUS_INVALID and L.TPD_ERR_TIMEOUT == STATUS_TIMEOUT


def test_graph_replay_after_smaller_launches_of_the_same_kernels(tpd):
    """Kernel nodes captured in a CUDA graph keep the dynamic shared-memory size
    of their capture.  A kernel's shared-memory limit that later calls lower to
    their own, smaller size (2^10-element tiles of the same pass kernels) would
    make the replayed nodes -- or a profiler relaunching them one by one --
    fail to launch; the library only ever raises the limit to each kernel's
    largest launch.  The replay must run and give the captured calls' results."""
    ns = [10, 10, 9, 8, 7]
    mats = [gpu(synth.general(n, seed=9900 + i)) for i, n in enumerate(ns)]
    want = [tpd.decompose(m) for m in mats]
    work = [m.clone() for m in mats]
    for prec_form in (0, 2):                          # per (n, pass) launches, one persistent launch
        batch = tpd.Batch(work, variant=prec_form)
        batch.decompose()                            # kernel attributes set outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            batch.decompose()
        # the same pass kernels launched with 2^10-element tiles (a quarter of the
        # captured shared memory), and whole small matrices
        for n in (8, 9, 10):
            tpd.decompose(gpu(synth.general(n, seed=n)), tile_bits=10)
        tpd.decompose(gpu(synth.general(3, seed=3)))
        torch.cuda.synchronize()
        for _ in range(2):
            for w, m in zip(work, mats):
                w.copy_(m)
            g.replay()
            torch.cuda.synchronize()
            for w, r in zip(work, want):
                assert torch.equal(w, r)
        assert batch.status() == STATUS_OK
