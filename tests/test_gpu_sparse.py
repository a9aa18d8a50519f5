"""GPU: sparse input (COO) -- the level-by-level decomposition of nonzero
entries with zero pruning -- against the CPU oracle on the dense matrix, on
planted Hamiltonians (exact), and its capacity handling."""
import numpy as np
import pytest

import oracle
from paper_2310_13421_gb300 import synth
from _helpers import assert_close, assert_exact

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def coo(H):
    r, c = np.nonzero(H)
    t = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
    return t(r.astype(np.int32), torch.int32), t(c.astype(np.int32), torch.int32), t(H[r, c], torch.complex128)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [2, 6, 10, 12])
def test_planted_heisenberg_exact(tpd, n):
    J, h = synth.heisenberg_params(n, seed=9700 + n)
    H = synth.heisenberg(n, J, h)
    want = sorted((synth.string_index(t), v) for t, v in synth.heisenberg_terms(n, J, h).items())
    s, w = tpd.decompose_coo(*coo(H), n)
    assert host(s).tolist() == [k for k, _ in want]
    assert_exact(host(w), np.array([v for _, v in want], dtype=np.complex128))


def test_tfim_eq7(tpd):
    n, J, g = 9, 0.75, 1.25
    H = synth.tfim(n, J, g)
    want = sorted((synth.string_index(t), v) for t, v in synth.tfim_terms(n, J, g).items())
    s, w = tpd.decompose_coo(*coo(H), n)
    assert len(want) == 2 * n - 1
    assert host(s).tolist() == [k for k, _ in want]
    assert_exact(host(w), np.array([v for _, v in want], dtype=np.complex128))


@pytest.mark.parametrize("n,m", [(5, 40), (8, 600), (9, 3000)])
def test_random_sparse_matches_oracle(tpd, n, m):
    rng = np.random.default_rng(9710 + n)
    N = 2 ** n
    r = rng.integers(0, N, size=m)
    c = rng.integers(0, N, size=m)
    v = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    H = np.zeros((N, N), dtype=np.complex128)
    np.add.at(H, (r, c), v)                        # duplicates add up
    want = oracle.coeffs_fwht(H)
    rows = torch.from_numpy(r.astype(np.int32)).cuda()
    cols = torch.from_numpy(c.astype(np.int32)).cuda()
    vals = torch.from_numpy(v).cuda()
    s, w = tpd.decompose_coo(rows, cols, vals, n)
    s = host(s)
    nz = np.flatnonzero(np.abs(want) > 1e-14 * np.max(np.abs(want)))
    assert s.tolist() == nz.tolist()
    assert_close(host(w), want[nz], 1e-12, "sparse n=%d" % n)


def test_diagonal_and_empty_and_capacity(tpd):
    n = 7
    d = np.arange(1, 2 ** n + 1, dtype=np.float64)
    s, w = tpd.decompose_coo(*coo(np.diag(d).astype(np.complex128)), n)
    digits = host(s)
    for b in range(n):
        assert np.all(np.isin((digits >> (2 * b)) & 3, (0, 3)))      # only I and Z factors
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    s0, w0 = tpd.decompose_coo(e, e, torch.empty(0, dtype=torch.complex128, device="cuda"), 5)
    assert s0.numel() == 0
    from paper_2310_13421_gb300 import _lib as L
    with pytest.raises(L.TPDError):
        tpd.decompose_coo(*coo(np.diag(d).astype(np.complex128)), n, max_entries=8)
    # the default sizing grows on demand and still gives the full list
    J, h = synth.heisenberg_params(8, seed=9720)
    H = synth.heisenberg(8, J, h)
    s1, _ = tpd.decompose_coo(*coo(H), 8, max_entries=None)
    assert s1.numel() == 3 * 7 + 8
