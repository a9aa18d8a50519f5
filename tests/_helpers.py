"""Test-side helpers: layout conversion and tolerance checks (independent of
the package's own helpers)."""
import numpy as np

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def rc_positions(n):
    """pos[s] = flat RC index of string s (t_j = 2 r_{n-j} + c_{n-j})."""
    s = np.arange(4 ** n, dtype=np.int64)
    r = np.zeros_like(s)
    c = np.zeros_like(s)
    for beta in range(n):
        t = (s >> (2 * beta)) & 3
        r |= (t >> 1) << beta
        c |= (t & 1) << beta
    return (r << n) | c


def to_string_order(rc, n):
    return np.asarray(rc).reshape(-1)[rc_positions(n)]


def rc_index_of_xz(x, z, n):
    """Flat RC index of the string with X-mask x, Z-mask z (arrays)."""
    x = np.asarray(x, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    # per bit: (x,z) -> t: (0,0) I=0 (r0,c0); (1,0) X=1 (r0,c1); (1,1) Y=2 (r1,c0); (0,1) Z=3 (r1,c1)
    r = z                      # row bit set for Y, Z
    c = x ^ z                  # column bit set for X, Z
    return (r << n) | c


def rel_err(got, want):
    want = np.asarray(want)
    den = np.linalg.norm(want.reshape(-1))
    return np.linalg.norm((np.asarray(got) - want).reshape(-1)) / (den if den else 1.0)


def assert_close(got, want, rtol, what=""):
    """Normwise ||got-want|| <= rtol ||want|| and elementwise <= rtol * max|want|."""
    got = np.asarray(got).reshape(-1)
    want = np.asarray(want).reshape(-1)
    e = rel_err(got, want)
    m = np.max(np.abs(got - want)) / max(np.max(np.abs(want)), 1e-300)
    assert e <= rtol and m <= rtol, "%s normwise %.3e elementwise %.3e > %.1e" % (what, e, m, rtol)


def assert_exact(got, want, what=""):
    got = np.asarray(got).reshape(-1)
    want = np.asarray(want).reshape(-1)
    bad = np.flatnonzero(got != want)  # +0 == -0
    assert bad.size == 0, "%s: %d mismatches, first at %d: %r vs %r" % (
        what, bad.size, bad[0], got[bad[0]], want[bad[0]])
