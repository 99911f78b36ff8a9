"""Pins for the function approximations of App. D.2 (oracle/approx.py).

Each function is checked against a closed form of the method it implements
(not against its own code): the limit approximation
lexp(x) = (1 + x/256)^256, the Newton-Raphson fixed points 1/x and 1/sqrt(x),
the Householder fixed point of ln with lexp inside (256 (1 - x^(-1/256))),
the Maclaurin polynomial, and exact max.  Tolerances come from fixed-point
error bounds:
  * a two-party truncation is off by 0..2 ulp (ulp = 2^-16): each share is
    floored, and the floors of the shares of v sum to floor(v) or floor(v) - 1;
  * exp: the first truncation (x / 256) is amplified 256-fold and the one
    after squaring k by 2^(8-k), so |lexp~/lexp - 1| <= 2 ulp (256 + sum_k
    2^(8-k) / y_k) ~ 0.019 on [-4, 2] (y_k >= 0.0177 there);
  * everything built on exp inherits that relative bound.
"""
import math

import numpy as np
import pytest

from oracle import approx, fixed, sharing

ULP = 2.0 ** -16
EXP_REL = 0.019


def _shared(v, op=1):
    return sharing.share(fixed.encode(np.asarray(v, dtype=np.float64)), 2, 0, 1, op)


def _reveal(X):
    return fixed.decode(sharing.reveal(X))


def lexp(x):
    return (1 + np.asarray(x) / 256.0) ** 256


def test_exp_limit_approximation():
    x = np.linspace(-4, 2, 400)
    got = _reveal(approx.exp(_shared(x), 1, approx.OpIds(100)))
    assert np.all(np.abs(got / lexp(x) - 1) < EXP_REL)
    # near 0 the limit approximation itself is within x^2/512 of e^x
    z = np.linspace(-1, 1, 101)
    g = _reveal(approx.exp(_shared(z), 2, approx.OpIds(100)))
    assert np.all(np.abs(g / np.exp(z) - 1) < EXP_REL + 1 / 512)


def test_reciprocal_positive_newton_raphson():
    x = np.linspace(0.1, 20, 400)
    got = _reveal(approx.reciprocal_pos(_shared(x), 1, approx.OpIds(200)))
    # NR converges to 1/x from y0 in (0, 2/x); a few ulps of truncation remain
    assert np.allclose(got, 1 / x, rtol=2e-3, atol=8 * ULP)


def test_reciprocal_either_sign():
    x = np.concatenate([np.linspace(-20, -0.1, 200), np.linspace(0.1, 20, 200)])
    got = _reveal(approx.reciprocal(_shared(x), 1, approx.OpIds(200)))
    assert np.allclose(got, 1 / x, rtol=2e-3, atol=8 * ULP)


def test_sigmoid_and_tanh():
    x = np.linspace(-8, 8, 401)
    s = _reveal(approx.sigmoid(_shared(x), 1, approx.OpIds(300)))
    # sigma(|x|) with lexp; |d sigma / d e| <= 1/4, so a relative exp error of
    # EXP_REL moves sigma by at most EXP_REL / 4
    lsig = 1 / (1 + lexp(-np.abs(x)))
    ref = np.where(x < 0, 1 - lsig, lsig)
    assert np.max(np.abs(s - ref)) < EXP_REL / 4 + 8 * ULP
    assert np.max(np.abs(s - 1 / (1 + np.exp(-x)))) < EXP_REL / 4 + 2e-3
    assert np.all(s[x < 0] < 0.5) and np.all(s[x > 0] > 0.5)
    t = _reveal(approx.tanh(_shared(x / 4), 1, approx.OpIds(400)))
    assert np.max(np.abs(t - np.tanh(x / 4))) < 2 * (EXP_REL / 4 + 2e-3)


def test_erf_maclaurin():
    x = np.linspace(-1, 1, 201)
    got = _reveal(approx.erf(_shared(x), 1, approx.OpIds(500)))
    ref = np.array([math.erf(v) for v in x])
    # remainder <= 2/sqrt(pi) / (9! 19) ~ 1.6e-7; nine truncated products and
    # nine truncated coefficient products at <= 2 ulp each, times coefficients <= 1.13
    assert np.max(np.abs(got - ref)) < 1e-3
    assert np.allclose(got, -got[::-1], atol=64 * ULP)     # odd function


def test_inv_sqrt_and_sqrt():
    x = np.linspace(0.01, 100, 500)
    y = _reveal(approx.inv_sqrt(_shared(x), 1, approx.OpIds(600)))
    # last step: t = x y^2 carries x * 2 ulp from y^2's truncation, and
    # y (3 - t) / 2 turns it into a relative error of t's error / 2 <= 100 ulp
    assert np.all(np.abs(y * np.sqrt(x) - 1) < 2e-3 + 200 * ULP)
    r = _reveal(approx.sqrt(_shared(x), 2, approx.OpIds(700)))
    assert np.all(np.abs(r / np.sqrt(x) - 1) < 2e-3 + 200 * ULP)


def test_log_householder_fixed_point():
    x = np.exp(np.linspace(np.log(1e-2), np.log(100), 300))
    got = _reveal(approx.log(_shared(x), 1, approx.OpIds(800)))
    # with lexp inside, h = 1 - x lexp(-y) vanishes at y* = 256 (1 - x^(-1/256));
    # an exp error of EXP_REL shifts h, hence y, by at most EXP_REL
    ystar = 256 * (1 - x ** (-1 / 256))
    assert np.max(np.abs(got - ystar)) < EXP_REL
    assert np.max(np.abs(got - np.log(x))) < EXP_REL + np.log(100) ** 2 / 512 + 1e-3


def test_max_lastdim_exact():
    rng = np.random.default_rng(4)
    for m in (1, 2, 3, 7, 8, 197):
        v = rng.integers(-(1 << 40), 1 << 40, (5, m))
        X = sharing.share(v.astype(np.int64).view(np.uint64), 2, 0, 1, 7)
        got = sharing.reveal(approx.max_lastdim(X, 1, approx.OpIds(1000))).view(np.int64)
        assert np.array_equal(got, v.max(axis=-1))


def test_softmax():
    rng = np.random.default_rng(0)
    v = rng.normal(0, 2, (6, 197))
    got = _reveal(approx.softmax(_shared(v), 1, approx.OpIds(900)))
    e = lexp(v - v.max(-1, keepdims=True))
    ref = e / e.sum(-1, keepdims=True)
    # numerator and denominator each within EXP_REL; the reciprocal and the
    # final product add a few ulps
    assert np.all(np.abs(got - ref) <= 2.2 * EXP_REL * ref + 16 * ULP)
    assert np.allclose(got.sum(-1), 1, atol=2 * EXP_REL)
