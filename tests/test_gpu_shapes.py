"""Pass kernels compiled for fixed tile layouts against the same kernels
reading the layout from the run-time pass descriptor (variant 5).

The two forms apply the same operations to the same elements in the same
order, so every output bit must agree: finite random inputs at sizes whose
default plans use each compiled layout, all-zero tiles (zero skipping),
Inf/NaN tiles (the IEEE fallback), the batched call, and the composition.
Correctness against the oracle is covered by the other GPU tests, which run
the compiled layouts by default.
"""
import numpy as np
import pytest

from paper_2310_13421_gb300 import _lib as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tpd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_13421_gb300 as pkg
    pkg.build()
    return pkg


def rand_matrix(n, dtype, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    real = torch.float64 if dtype == torch.complex128 else torch.float32
    N = 1 << n
    re = torch.randn(N, N, generator=g, device="cuda", dtype=real)
    im = torch.randn(N, N, generator=g, device="cuda", dtype=real)
    return torch.complex(re, im)


def bits(t):
    real = t.real.dtype
    return t.view(real).view(torch.int64 if real == torch.float64 else torch.int32)


def assert_same_bits(a, b, what):
    torch.cuda.synchronize()
    ba, bb = bits(a), bits(b)
    bad = (ba != bb).nonzero()
    assert bad.numel() == 0, "%s: %d words differ, first at %s" % (what, bad.shape[0], bad[0].tolist())


def shapes_of(n, dtype, prec):
    desc = L.tpd_plan_describe(n, dtype, L.options(precision=prec))[1]
    return [int(tok.split("=")[1]) for tok in desc.split() if tok.startswith("shape=")]


CASES = [
    # (storage, precision, n): every compiled layout, each role of the fixed point
    ("c128", "fixed", 9), ("c128", "fixed", 10), ("c128", "fixed", 11), ("c128", "fixed", 12), ("c128", "fixed", 13),
    ("c128", "fixed", 14), ("c128", "fixed", 15),
    ("c64", "plain", 11), ("c64", "plain", 12), ("c64", "plain", 13), ("c64", "plain", 14), ("c64", "plain", 15),
    ("c64", "fixed", 11), ("c64", "fixed", 12), ("c64", "fixed", 13), ("c64", "fixed", 15),
    ("c64", "compensated", 12), ("c64", "compensated", 13), ("c64", "compensated", 14),
    ("c64", "compensated", 15),
]


@pytest.mark.parametrize("storage,precision,n", CASES)
def test_compiled_layouts_match_runtime_layouts(tpd, storage, precision, n):
    dtype = torch.complex128 if storage == "c128" else torch.complex64
    code = L.TPD_C128 if storage == "c128" else L.TPD_C64
    prec = {"fixed": L.TPD_PREC_FIXED, "plain": L.TPD_PREC_PLAIN,
            "compensated": L.TPD_PREC_COMPENSATED}[precision]
    assert any(s >= 0 for s in shapes_of(n, code, prec)), "no compiled layout in this plan"
    A = rand_matrix(n, dtype, 31000 + n)
    got = tpd.decompose(A, precision=precision)
    want = tpd.decompose(A, precision=precision, variant=5)
    assert_same_bits(got, want, "%s %s n=%d" % (storage, precision, n))
    del got, want, A
    torch.cuda.empty_cache()


@pytest.mark.parametrize("storage,precision",
                         [("c128", "fixed"), ("c64", "plain"), ("c64", "compensated"), ("c64", "fixed")])
def test_zero_tiles_and_non_finite_tiles(tpd, storage, precision):
    dtype = torch.complex128 if storage == "c128" else torch.complex64
    n = 13
    A = rand_matrix(n, dtype, 31100)
    N = 1 << n
    A[: N // 2, : N // 4] = 0                           # whole tiles of zeros in every pass
    A[N // 2:, N // 2:: 7] = 0
    A[5, 9] = complex(float("inf"), 1.0)                # Inf / NaN tiles take the IEEE path
    A[N - 3, 17] = complex(0.0, float("nan"))
    for skip in (False, True):
        got = tpd.decompose(A, precision=precision, skip_zero=skip)
        want = tpd.decompose(A, precision=precision, skip_zero=skip, variant=5)
        assert_same_bits(got, want, "%s %s skip=%s" % (storage, precision, skip))


def test_batched_and_composition(tpd):
    mats = [rand_matrix(n, torch.complex128, 31200 + i) for i, n in enumerate([9, 10, 12, 9, 12, 10])]
    got = tpd.decompose_batched(mats)
    want = tpd.decompose_batched(mats, variant=5)
    for i, (g, w) in enumerate(zip(got, want)):
        assert_same_bits(g, w, "batched matrix %d" % i)
    C = rand_matrix(13, torch.complex128, 31300)
    assert_same_bits(tpd.compose(C), tpd.compose(C, variant=5), "composition n=13")
