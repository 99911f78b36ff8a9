"""Exact pins for the function approximations of App. D.2 (oracle/approx.py).

With a single party every Beaver product is exact and the "two-party"
truncation of the one share is exactly floor(v / 2^f), so the oracle's result
for P = 1 is a deterministic fixed-point computation.  This file replays each
method step by step on plain Python integers -- the iteration formulas of
App. D.2 with the readings the build takes (n = 8 for the limit exp, 10
Newton-Raphson steps from the paper's initial values, K = 8 Maclaurin terms,
3 Householder steps of order 8, the initial value of the inverse square root),
one floor per truncated product -- written independently of the oracle, and
requires the oracle's P = 1 output to equal it word for word.  A dropped term,
a wrong constant, an iteration too many or too few, or a truncation by the
wrong number of bits all change the integers.  The two-party results are then
pinned by the closed-form bounds in test_oracle_approx.py.

Ring arithmetic: every intermediate is reduced to the signed 64-bit view, as
the shares are words of Z/2^64.
"""
import math

import numpy as np
import pytest

from oracle import approx, fixed, sharing

ONE = 1 << 16
M64 = 1 << 64


def w(v):
    """Signed view of v mod 2^64."""
    return (v + (1 << 63)) % M64 - (1 << 63)


def fl(v, f):
    """floor(s(v) / 2^f): the truncation of a single share."""
    return w(v) >> f


def prod(a, b, f=16):
    """Beaver product of two values, then truncation by f bits (f = 0: none)."""
    return fl(a * b, f) if f else w(a * b)


def code(c):
    """A public constant in fixed point: round half to even of c * 2^16."""
    return int(round(c * ONE))


# ---- the methods, on integers --------------------------------------------------------
def r_exp(x, n=8):
    y = w(fl(x, n) + ONE)                 # 1 + x / 2^n
    for _ in range(n):
        y = prod(y, y)                    # squared n times
    return y


def r_newton_recip(a, y, iters=10):
    """y <- y (2 - a y)."""
    for _ in range(iters):
        y = prod(y, w(2 * ONE - prod(a, y)))
    return y


def r_recip_pos(x):
    y0 = w(3 * r_exp(w(ONE // 2 - x)) + code(0.003))    # 3 e^(1/2 - x) + 0.003
    return r_newton_recip(x, y0)


def r_sign(x):
    c = 1 if w(x) < 0 else 0
    sgn = 1 - 2 * c
    return c, sgn, w(x * sgn)


def r_recip(x):
    _, sgn, ax = r_sign(x)
    return w(r_recip_pos(ax) * sgn)


def r_sigmoid(x):
    c, _, ax = r_sign(x)
    s = r_newton_recip(w(r_exp(w(-ax)) + ONE), code(0.75))    # 1 / (1 + e^-|x|)
    return w(c * w(w(ONE - s) - s) + s)                        # c ? 1 - s : s


def r_tanh(x):
    return w(2 * r_sigmoid(w(2 * x)) - ONE)


def r_erf(x, terms=8):
    x2 = prod(x, x)
    p = x
    acc = fl(code(2 / math.sqrt(math.pi)) * x, 16)
    for k in range(1, terms + 1):
        p = prod(p, x2)                                       # x^(2k+1)
        c = 2 / math.sqrt(math.pi) * (-1) ** k / (math.factorial(k) * (2 * k + 1))
        acc = w(acc + fl(code(c) * p, 16))
    return acc


def r_inv_sqrt(x, iters=10):
    g = r_exp(fl(-x, 4))                                      # e^(-x/16)
    e = g
    for _ in range(4):
        e = prod(e, e)                                        # e^(-x)
    y = w(w(3 * e + code(0.05)) + fl(code(0.3) * g, 16))
    for _ in range(iters):
        t = prod(x, prod(y, y))
        y = prod(y, w(3 * ONE - t), 17)                       # y (3 - x y^2) / 2
    return y


def r_sqrt(x):
    return prod(x, r_inv_sqrt(x))


def r_log(x, iters=3, order=8):
    y = w(fl(code(1 / 120) * x, 16) + w(3 * ONE - 20 * r_exp(w(-2 * x - ONE))))
    for _ in range(iters):
        h = w(ONE - prod(x, r_exp(w(-y))))
        p, s = h, h
        for k in range(2, order + 1):
            p = prod(p, h)
            s = w(s + fl(code(1 / k) * p, 16))
        y = w(y - s)
    return y


def r_softmax_row(row):
    mx = max(w(v) for v in row)
    e = [r_exp(w(v - mx)) for v in row]
    r = r_recip_pos(w(sum(e)))
    return [prod(v, r) for v in e]


# ---- pins ------------------------------------------------------------------------------
def _one_party(vals):
    enc = fixed.encode(np.asarray(vals, dtype=np.float64))
    return sharing.share(enc, 1, 0, 1, 3), [int(v) for v in enc.view(np.int64)]


def _ints(shares):
    return [int(v) for v in sharing.reveal(shares).view(np.int64).ravel()]


CASES = {
    "exp": (approx.exp, r_exp, np.concatenate([np.linspace(-8, 3, 160), [0.0, -2 ** -16]])),
    "reciprocal_pos": (approx.reciprocal_pos, r_recip_pos, np.linspace(0.05, 30, 120)),
    "reciprocal": (approx.reciprocal, r_recip,
                   np.concatenate([np.linspace(-30, -0.05, 60), np.linspace(0.05, 30, 60)])),
    "sigmoid": (approx.sigmoid, r_sigmoid, np.concatenate([np.linspace(-12, 12, 121), [0.0]])),
    "tanh": (approx.tanh, r_tanh, np.linspace(-5, 5, 101)),
    "erf": (approx.erf, r_erf, np.linspace(-1.5, 1.5, 121)),
    "inv_sqrt": (approx.inv_sqrt, r_inv_sqrt, np.geomspace(0.01, 100, 100)),
    "sqrt": (approx.sqrt, r_sqrt, np.geomspace(0.01, 100, 100)),
    "log": (approx.log, r_log, np.geomspace(0.01, 100, 100)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_party_oracle_equals_integer_replay(name):
    fn, replay, vals = CASES[name]
    X, xs = _one_party(vals)
    got = _ints(fn(X, 1, approx.OpIds(100)))
    assert got == [replay(v) for v in xs], name


def test_one_party_max_and_softmax_equal_integer_replay():
    rng = np.random.default_rng(4)
    for m in (1, 2, 3, 7, 16, 33):
        rows = rng.normal(0, 2, (5, m))
        X, xs = _one_party(rows.ravel())
        X = X.reshape(1, 5, m)
        xs = [xs[r * m:(r + 1) * m] for r in range(5)]
        assert _ints(approx.max_lastdim(X, 1, approx.OpIds(10))) == [max(r) for r in xs]
        got = _ints(approx.softmax(X, 1, approx.OpIds(10)))
        assert got == [v for r in xs for v in r_softmax_row(r)], m


def test_replay_detects_planted_slips():
    """The pin is sensitive: the oracle run with a different method parameter
    (an exp squaring fewer, Newton steps fewer, a Maclaurin term fewer, a
    Householder step fewer) no longer equals the replay of the stated method.
    Two slips are invisible by the method's own arithmetic and are not used:
    the 8th Maclaurin coefficient of erf, 2/sqrt(pi) / (8! 17) = 1.6e-6, encodes
    to 0 at 2^16, and Newton-Raphson for 1/x has converged to the last bit
    after 9 of its 10 steps."""
    X, xs = _one_party(np.linspace(0.1, 3, 40))
    assert code(2 / math.sqrt(math.pi) / (math.factorial(8) * 17)) == 0
    assert _ints(approx.exp(X, 1, approx.OpIds(100), iters=7)) != [r_exp(v) for v in xs]
    assert _ints(approx.erf(X, 1, approx.OpIds(100), terms=6)) != [r_erf(v) for v in xs]
    assert _ints(approx.log(X, 1, approx.OpIds(100), iters=2)) != [r_log(v) for v in xs]
    assert _ints(approx.inv_sqrt(X, 1, approx.OpIds(100), iters=9)) != [r_inv_sqrt(v) for v in xs]
    X2, xs2 = _one_party(np.linspace(0.1, 30, 40))
    assert _ints(approx.reciprocal_pos(X2, 1, approx.OpIds(100), iters=8)) != \
        [r_recip_pos(v) for v in xs2]


def test_replay_matches_the_closed_forms():
    """The integer replays themselves approximate what App. D.2 says they
    compute (so a replay slip cannot pass by matching an oracle slip)."""
    d = lambda v: v / ONE
    for x in np.linspace(-4, 2, 25):
        assert abs(d(r_exp(code(x))) / (1 + x / 256) ** 256 - 1) < 0.01
    for x in np.linspace(0.1, 20, 25):
        assert abs(d(r_recip_pos(code(x))) * x - 1) < 2e-3 + 8 * x / ONE
    for x in np.linspace(-6, 6, 25):
        ls = 1 / (1 + (1 - abs(x) / 256) ** 256)
        assert abs(d(r_sigmoid(code(x))) - (ls if x >= 0 else 1 - ls)) < 3e-3
    for x in np.linspace(-1, 1, 21):
        assert abs(d(r_erf(code(x))) - math.erf(x)) < 5e-4
    for x in np.geomspace(0.01, 100, 21):
        assert abs(d(r_inv_sqrt(code(x))) * math.sqrt(x) - 1) < 3e-3
        fp = 256 * (1 - x ** (-1 / 256))      # fixed point of the iteration with lexp inside
        assert abs(d(r_log(code(x))) - fp) < 0.02 * max(1.0, abs(fp))
