"""Full-size parity for the five workloads, in the launch configuration the
benchmark times: sampled outputs the oracle computes X-row by X-row (all 2^n
Z-masks of a chosen X-mask in O(n 2^n)), plus invariants that hold at any
size (Parseval, exact planted recovery, Hermitian => real)."""
import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import U32, assert_close, assert_exact, rc_index_of_xz, rc_positions, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def sample_rows(A_host, out_gpu, n, xs):
    """Compare the GPU result (RC layout, on device) on the X-rows xs."""
    want = oracle.coeffs_xrows(A_host, np.asarray(xs, dtype=np.uint64))
    z = np.arange(2 ** n, dtype=np.int64)
    idx = np.concatenate([rc_index_of_xz(np.full_like(z, x), z, n) for x in xs])
    got = out_gpu.reshape(-1)[torch.from_numpy(idx).cuda()].cpu().numpy()
    return got, want.reshape(-1)


def parseval(A_gpu, C_gpu, n):
    a = torch.sum(A_gpu.real.double() ** 2 + A_gpu.imag.double() ** 2).item()
    c = torch.sum(C_gpu.real.double() ** 2 + C_gpu.imag.double() ** 2).item() * 2 ** n
    return abs(a - c) / a


def test_config_n14_dense_c128(tpd):
    n = 14
    A = synth.hermitian(n, seed=1002)
    Ag = torch.from_numpy(A).cuda()
    rng = np.random.default_rng(14)
    xs = [0, 1, 2 ** n - 1, 2 ** (n - 1)] + list(rng.integers(0, 2 ** n, size=28))
    for prec in ("fixed", "plain"):
        C = tpd.decompose(Ag, precision=prec)
        got, want = sample_rows(A, C, n, xs)
        assert_close(got, want, 1e-12, "n=14 " + prec)
        assert parseval(Ag, C, n) <= 1e-12
        # Hermitian input: real weights, exactly (both arithmetics are odd-symmetric)
        assert torch.count_nonzero(C.imag).item() == 0
        del C
    # zero skip on a dense input changes nothing
    C1 = tpd.decompose(Ag)
    C2 = tpd.decompose(Ag, skip_zero=True)
    assert torch.equal(C1, C2)


def test_config_n14_planted_heisenberg(tpd):
    n = 14
    for dy in (synth.DYADIC_BITS, None):
        J, h = synth.heisenberg_params(n, seed=1102, dyadic_bits=dy)
        H = torch.from_numpy(synth.heisenberg(n, J, h)).cuda()
        terms = synth.heisenberg_terms(n, J, h)
        assert len(terms) == 3 * (n - 1) + n
        pos = rc_positions(n)
        idx = torch.tensor([int(pos[synth.string_index(t)]) for t in terms], device="cuda")
        vals = torch.tensor([complex(v) for v in terms.values()], dtype=torch.complex128, device="cuda")
        for prec in ("fixed", "plain"):
            C = tpd.decompose(H, precision=prec, skip_zero=True).reshape(-1)
            if dy is not None:  # dyadic couplings: every weight exact, the other 4^n - 53 exactly zero
                want = torch.zeros_like(C)
                want[idx] = vals
                assert torch.equal(C, want)
            else:
                assert torch.max(torch.abs(C[idx] - vals)).item() <= 1e-12 * torch.max(torch.abs(vals)).item()
                C[idx] = 0
                assert torch.max(torch.abs(C)).item() <= 1e-12 * torch.max(torch.abs(vals)).item()
            del C


def test_config_n15_c64_plain_and_compensated(tpd):
    n = 15
    A64 = synth.hermitian(n, seed=1003, dtype=np.complex64)
    Ag = torch.from_numpy(A64).cuda()
    A_up = A64.astype(np.complex128)
    rng = np.random.default_rng(15)
    xs = [0, 2 ** n - 1] + list(rng.integers(0, 2 ** n, size=14))
    from paper_2310_13421_gb300 import _lib as L
    P = L.tpd_plan_describe(n, 1, L.options(precision=2))[0]
    errs = {}
    for prec in ("plain", "compensated"):
        C = tpd.decompose(Ag, precision=prec)
        got, want = sample_rows(A_up, C, n, xs)
        errs[prec] = rel_err(got.astype(np.complex128), want)
        del C
    assert errs["plain"] <= n * U32
    assert errs["compensated"] <= (P + 1) * U32
    assert errs["compensated"] < errs["plain"]
    # the complex64 block fixed point: exact sums, one rounding per pass (its own plan: 3 passes here)
    Pf = L.tpd_plan_describe(n, 1, L.options(precision=3))[0]
    C = tpd.decompose(Ag, precision="fixed")
    got, want = sample_rows(A_up, C, n, xs)
    del C
    assert rel_err(got.astype(np.complex128), want) <= Pf * U32 / (1 - Pf * U32)
    # against the complex128 decomposition of the same (upcast) matrix on the GPU
    C128 = tpd.decompose(Ag.to(torch.complex128))
    Cc = tpd.decompose(Ag, precision="compensated").to(torch.complex128)
    e = (torch.linalg.vector_norm(Cc - C128) / torch.linalg.vector_norm(C128)).item()
    assert e <= 1e-6


def test_n15_complex128_sampled_rows_and_planted_chain(tpd):
    """n = 15 in complex128: the plan mixes 2^12- and 2^13-element tiles (the
    middle pass of 5 levels needs the larger tile); sampled X-rows against
    the oracle for a random Hermitian matrix, and the planted Heisenberg
    chain's weights exactly."""
    n = 15
    from paper_2310_13421_gb300 import _lib as L
    desc = L.tpd_plan_describe(n, 0, L.options())[1]
    assert "D=13" in desc and "D=12" in desc
    A = synth.hermitian(n, seed=1015)
    Ag = torch.from_numpy(A).cuda()
    rng = np.random.default_rng(1015)
    xs = [0, 2 ** n - 1, 2 ** (n - 1)] + list(rng.integers(0, 2 ** n, size=9))
    for prec in ("fixed", "plain"):
        C = tpd.decompose(Ag, precision=prec)
        got, want = sample_rows(A, C, n, xs)
        assert_close(got, want, 1e-12, "n=15 " + prec)
        assert parseval(Ag, C, n) <= 1e-12
        del C
    del Ag
    J, h = synth.heisenberg_params(n, seed=1016)
    H = torch.zeros((1 << n, 1 << n), dtype=torch.complex128, device="cuda")
    synth.heisenberg_into(H, n, J, h)
    tpd.decompose(H, inplace=True)
    s, w = tpd.nonzero_list(H)
    want = sorted((synth.string_index(t), v) for t, v in synth.heisenberg_terms(n, J, h).items())
    assert s.cpu().tolist() == [k for k, _ in want]
    assert np.array_equal(w.cpu().numpy(), np.array([v for _, v in want], dtype=np.complex128))
    del H
    torch.cuda.empty_cache()


def test_config_batch_4096(tpd):
    ns = synth.batch_sizes(4096, seed=1004)
    mats = [torch.empty((2 ** int(n), 2 ** int(n)), dtype=torch.complex128, device="cuda") for n in ns]
    host = {}
    check = set(np.random.default_rng(4).choice(4096, size=48, replace=False).tolist())
    for i, (n, m) in enumerate(zip(ns, mats)):
        a = synth.hermitian(int(n), seed=100000 + i)
        m.copy_(torch.from_numpy(a))
        if i in check:
            host[i] = a
    orig = [m.clone() for m in mats]
    batch = tpd.Batch(mats)
    g = torch.cuda.CUDAGraph()
    batch.decompose()                 # warm-up outside capture
    for m, o in zip(mats, orig):
        m.copy_(o)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        batch.decompose()
    g.replay()
    torch.cuda.synchronize()
    for i in check:
        n = int(ns[i])
        got = mats[i].cpu().numpy().reshape(-1)[rc_positions(n)]
        assert_close(got, oracle.coeffs_fwht(host[i]), 1e-12, "batch item %d n=%d" % (i, n))
    worst = max(parseval(o, m, int(n)) for o, m, n in zip(orig, mats, ns))
    assert worst <= 1e-12


def test_config_n12_autograd(tpd):
    n = 12
    A = synth.hermitian(n, seed=1005)
    w = synth.loss_weights(n, seed=1105)
    w_rc = np.empty(4 ** n)
    w_rc[rc_positions(n)] = w
    W = torch.from_numpy(w_rc).cuda().reshape(2 ** n, 2 ** n)
    At = torch.from_numpy(A).cuda().requires_grad_(True)

    def loss(M):
        c = tpd.tpd(M)
        return (W * (c.real ** 2 + c.imag ** 2)).sum()

    L0 = loss(At)
    L0.backward()
    G = At.grad.detach()
    assert_close(G.cpu().numpy(), oracle.grad_weighted_sq(A, w), 1e-12, "oracle gradient")
    # central differences on 64 distinct random entries (real and imaginary
    # direction each): L is quadratic, so exact up to rounding
    rng = np.random.default_rng(12)
    flat = rng.choice(4 ** n, size=64, replace=False)
    hstep = 1e-2
    with torch.no_grad():
        base = torch.from_numpy(A).cuda()
        for f in flat:
            i, j = divmod(int(f), 2 ** n)
            for unit in (1.0, 1j):
                Ap = base.clone(); Ap[i, j] += hstep * unit
                Am = base.clone(); Am[i, j] -= hstep * unit
                fd = (loss(Ap) - loss(Am)).item() / (2 * hstep)
                an = G[i, j].real.item() if unit == 1.0 else G[i, j].imag.item()
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (i, j, unit, fd, an)
