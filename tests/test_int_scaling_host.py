"""CPU: the integer scalings by powers of two that the fp64 kernels use in
place of fp64 multiplies -- x / 2 and 2 x in the Gell-Mann levels, x 2^-K in
the fp64 Pauli passes -- transcribed step by step from the device routines
into numpy int64 arithmetic and compared bit for bit with the IEEE products
over the whole double range: normal numbers, subnormal results (rounded to
nearest even from the magnitude bits), zeros of both signs, overflow to Inf,
and Inf.  (NaN passes unchanged, so only its NaN-ness is compared.)  The GPU
tests check the kernels' outputs against the oracle; this checks the method
the kernels rely on at every boundary of the exponent range."""
import numpy as np
import pytest

SGN = np.int64(-0x8000000000000000)
MAG = np.int64(0x7FFFFFFFFFFFFFFF)
MANT = np.int64(0x000FFFFFFFFFFFFF)


def doubles(seed):
    g = np.random.default_rng(seed)
    with np.errstate(over="ignore"):                   # huge draws overflow to +-Inf: kept as inputs
        x = _draw(g)
    return x[~np.isnan(x)]


def _draw(g):
    x = np.concatenate([
        g.standard_normal(200000) * 10.0 ** g.integers(-324, 309, 200000),
        np.frombuffer(g.integers(0, 2 ** 63, 100000, dtype=np.int64).tobytes(), dtype=np.float64),
        np.frombuffer(g.integers(0, 2 ** 53, 20000, dtype=np.int64).tobytes(), dtype=np.float64),   # subnormals
        np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1e-323, 1.5e-323, 2.2250738585072014e-308,
                  -2.2250738585072014e-308, 2.225073858507201e-308, 4.450147717014403e-308,
                  8.98846567431158e307, 1.7976931348623157e308, -1.7976931348623157e308]),
    ])
    return np.concatenate([x, -x])


def ghalf(x):
    """x / 2: exponent field - 1 for a normal result; for e <= 1 the magnitude
    bits halved with ties to even; Inf and NaN unchanged"""
    b = x.view(np.int64)
    e = (b >> 52) & 0x7FF
    v = b & MAG
    sub = (b & SGN) | ((v >> 1) + ((v & (v >> 1)) & 1))
    return np.where((e >= 2) & (e < 0x7FF), b - (np.int64(1) << 52), np.where(e < 2, sub, b)).view(np.float64)


def gtwice(x):
    """2 x: the magnitude bits doubled for a subnormal input, exponent field
    + 1 for a normal one, Inf from the largest binade, Inf and NaN unchanged"""
    b = x.view(np.int64)
    e = (b >> 52) & 0x7FF
    s = b & SGN
    v = b & MAG
    return np.where(e == 0, s | (v << 1),
                    np.where(e < 0x7FE, b + (np.int64(1) << 52),
                             np.where(e == 0x7FE, s | np.int64(0x7FF0000000000000), b))).view(np.float64)


def mul_pow2_neg(x, sh):
    """x 2^-sh, 1 <= sh <= 11: exponent field - sh for a normal result, else the
    magnitude in units of 2^-1074 shifted right with round to nearest even"""
    b = x.view(np.int64)
    e = (b >> 52) & 0x7FF
    m = b & MANT
    v = np.where(e == 0, m, (m | (np.int64(1) << 52)) << np.clip(e - 1, 0, 10))
    q = v >> sh
    rem = v & ((np.int64(1) << sh) - 1)
    half = np.int64(1) << (sh - 1)
    q = q + ((rem > half) | ((rem == half) & ((q & 1) == 1))).astype(np.int64)
    out = np.where((e > sh) & (e < 0x7FF), b - (np.int64(sh) << 52), np.where(e == 0x7FF, b, (b & SGN) | q))
    return out.view(np.float64)


def same_bits(a, b):
    return np.array_equal(a.view(np.int64), b.view(np.int64))


def test_halving_and_doubling_are_the_ieee_products():
    x = doubles(1)
    with np.errstate(over="ignore"):
        assert same_bits(ghalf(x), x * 0.5)
        assert same_bits(gtwice(x), x * 2.0)


@pytest.mark.parametrize("sh", list(range(1, 12)))
def test_scaling_by_two_to_the_minus_k_is_the_ieee_product(sh):
    x = doubles(100 + sh)
    assert same_bits(mul_pow2_neg(x, sh), x * 2.0 ** -sh)


def test_nan_stays_nan():
    x = np.array([np.nan, -np.nan, np.frombuffer(np.int64(0x7FF0000000000001).tobytes(), dtype=np.float64)[0]])
    assert np.all(np.isnan(ghalf(x))) and np.all(np.isnan(gtwice(x))) and np.all(np.isnan(mul_pow2_neg(x, 6)))
