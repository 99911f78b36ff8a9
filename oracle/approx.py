"""Function approximations on shares (App. D.2), built from Beaver products,
truncation, public affine maps and comparisons.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Two parties, fixed point 2^16.  Every Beaver product or square of two scaled
values is followed by two-party truncation by 2^16; a product with an unscaled
0/1 or +-1 sharing is not truncated.  The k-th interactive step of a function
(a product, a square, a comparison, one level of a max tree) draws its dealer
material at op id base + 10 k (a comparison or ReLU uses op .. op + 3 of its
block, as everywhere else).

Readings (the paper fixes the methods, not every constant or order):
  * exp: the limit approximation (1 + x / 2^n)^(2^n) with n = 8; x / 2^n is a
    two-party truncation by n bits, then n squarings;
  * reciprocal: Newton-Raphson y <- y (2 - x y), 10 iterations, from
    y0 = 3 exp(0.5 - x) + 0.003 (the paper's default), for x > 0; for any sign
    1/x = sgn(x) / |x| with sgn(x) = 1 - 2 [x < 0] (an unscaled sharing);
  * sigmoid: sigma(|x|) = 1 / (1 + exp(-|x|)) by Newton-Raphson from y0 = 0.75
    (10 iterations), then sigma(x) = [x < 0] ? 1 - sigma(|x|) : sigma(|x|);
  * tanh(x) = 2 sigma(2x) - 1;
  * erf: the Maclaurin series with K = 8 (the paper's default), odd powers
    built by repeated products with x^2;
  * inverse square root: y <- y (3 - x y^2) / 2 (the /2 folded into the last
    product's truncation, by 17 bits), 10 iterations.  The paper gives no
    initial value; the oracle uses y0 = 3 g^16 + 0.3 g + 0.05 with
    g = exp(-x / 16) (g^16 = exp(-x) by four more squarings), which keeps
    y0 sqrt(x) within (0.3, 1.6), inside the convergence interval (0, sqrt 3),
    for x in [0.01, 100]; sqrt(x) = x * x^(-1/2);
  * log: Householder iterations of degree 8, h = 1 - x exp(-y),
    y <- y - sum_{k=1}^{8} h^k / k, 3 iterations, from
    y0 = x / 120 - 20 exp(-2x - 1) + 3 (the paper's defaults); powers of h by
    successive products;
  * max over the last axis: a tree of max(a, b) = b + ReLU(a - b) over
    adjacent pairs, one ReLU per level over all pairs of the level;
  * softmax over the last axis: e = exp(x - max(x)), s = sum(e) (local),
    softmax = e * reciprocal(s) with the positive-input reciprocal (s >= 1).
"""
import math

import numpy as np

from . import beaver, compare, dealer, truncation
from .beaver import affine
from .resnet import relu_shares

U64 = np.uint64
FRAC = 16
ONE = 1 << FRAC


class OpIds:
    """Consecutive op-id blocks of 10 for the interactive steps of a function."""

    def __init__(self, base):
        self.next_id = base

    def take(self):
        op = self.next_id
        self.next_id += 10
        return op


def enc(c):
    """Public real -> fixed-point integer (rint, ties to even)."""
    return int(np.rint(c * ONE))


def _add(x, y):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=U64) + np.asarray(y, dtype=U64)


def _sub(x, y):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=U64) - np.asarray(y, dtype=U64)


def mul(x, y, seed, ops, trunc_bits=FRAC):
    """Elementwise Beaver product (triple at the next op id), then truncation."""
    x = np.asarray(x, dtype=U64)
    P = x.shape[0]
    n = x[0].size
    A, B, C = dealer.mul_triple(P, n, seed, ops.take())
    z = beaver.beaver_mul(x.reshape(P, n), np.asarray(y, dtype=U64).reshape(P, n), A, B, C)
    z = z.reshape(x.shape)
    return truncation.truncate(z, trunc_bits) if trunc_bits else z


def square(x, seed, ops):
    x = np.asarray(x, dtype=U64)
    P = x.shape[0]
    n = x[0].size
    A, B = dealer.square_pair(P, n, seed, ops.take())
    z = beaver.beaver_square(x.reshape(P, n), A, B).reshape(x.shape)
    return truncation.truncate(z, FRAC)


def exp(x, seed, ops, iters=8):
    y = affine(affine(x, 1, 0, trunc_bits=iters), 1, ONE)   # 1 + x / 2^iters
    for _ in range(iters):
        y = square(y, seed, ops)
    return y


def reciprocal_nr(x, y, seed, ops, iters=10):
    """Newton-Raphson y <- y (2 - x y) from the initial sharing y."""
    for _ in range(iters):
        t = mul(x, y, seed, ops)
        y = mul(y, affine(t, -1, 2 * ONE), seed, ops)
    return y


def reciprocal_pos(x, seed, ops, iters=10):
    """1 / x for x > 0, initial guess y0 = 3 exp(0.5 - x) + 0.003."""
    y0 = affine(exp(affine(x, -1, ONE // 2), seed, ops), 3, enc(0.003))
    return reciprocal_nr(x, y0, seed, ops, iters)


def sign_split(x, seed, ops):
    """([x < 0], sgn(x) = 1 - 2 [x < 0], |x| = sgn(x) x), all from one comparison."""
    x = np.asarray(x, dtype=U64)
    c = compare.ltz(x.reshape(x.shape[0], -1), seed, ops.take()).reshape(x.shape)
    sgn = affine(c, -2, 1)
    return c, sgn, mul(x, sgn, seed, ops, trunc_bits=0)


def reciprocal(x, seed, ops, iters=10):
    """1 / x = sgn(x) / |x| for either sign."""
    _, sgn, ax = sign_split(x, seed, ops)
    return mul(reciprocal_pos(ax, seed, ops, iters), sgn, seed, ops, trunc_bits=0)


def sigmoid(x, seed, ops, iters=10):
    c, _, ax = sign_split(x, seed, ops)
    d = affine(exp(affine(ax, -1, 0), seed, ops), 1, ONE)     # 1 + exp(-|x|)
    y0 = np.zeros_like(d)
    y0[0] = U64(enc(0.75))                                    # public 0.75 on party 0
    s = reciprocal_nr(d, y0, seed, ops, iters)                # sigma(|x|)
    c = c.reshape(c.shape[0], -1)
    P = c.shape[0]
    out = compare.mux(c, affine(s, -1, ONE).reshape(P, -1), s.reshape(P, -1), seed, ops.take())
    return out.reshape(s.shape)


def tanh(x, seed, ops):
    return affine(sigmoid(affine(x, 2, 0), seed, ops), 2, -ONE)


def erf(x, seed, ops, terms=8):
    """2/sqrt(pi) sum_{k=0}^{terms} (-1)^k x^(2k+1) / (k! (2k+1))."""
    x = np.asarray(x, dtype=U64)
    x2 = square(x, seed, ops)
    p = x
    acc = affine(x, enc(2 / math.sqrt(math.pi)), 0, trunc_bits=FRAC)
    for k in range(1, terms + 1):
        p = mul(p, x2, seed, ops)
        coef = 2 / math.sqrt(math.pi) * (-1) ** k / (math.factorial(k) * (2 * k + 1))
        acc = _add(acc, affine(p, enc(coef), 0, trunc_bits=FRAC))
    return acc


def inv_sqrt(x, seed, ops, iters=10):
    """x^(-1/2) for x > 0 by y <- y (3 - x y^2) / 2 from y0 = 3 g^16 + 0.3 g + 0.05."""
    g = exp(affine(x, -1, 0, trunc_bits=4), seed, ops)        # exp(-x / 16)
    e = g
    for _ in range(4):
        e = square(e, seed, ops)                              # exp(-x)
    y = _add(affine(e, 3, enc(0.05)), affine(g, enc(0.3), 0, trunc_bits=FRAC))
    for _ in range(iters):
        t = mul(x, square(y, seed, ops), seed, ops)
        y = mul(y, affine(t, -1, 3 * ONE), seed, ops, trunc_bits=FRAC + 1)
    return y


def sqrt(x, seed, ops, iters=10):
    return mul(x, inv_sqrt(x, seed, ops, iters), seed, ops)


def log(x, seed, ops, iters=3, order=8):
    """ln x for x > 0: Householder iterations of the given polynomial order."""
    x = np.asarray(x, dtype=U64)
    y = _add(affine(x, enc(1 / 120), 0, trunc_bits=FRAC),
             affine(exp(affine(x, -2, -ONE), seed, ops), -20, 3 * ONE))
    for _ in range(iters):
        h = affine(mul(x, exp(affine(y, -1, 0), seed, ops), seed, ops), -1, ONE)
        p = h
        s = h
        for k in range(2, order + 1):
            p = mul(p, h, seed, ops)
            s = _add(s, affine(p, enc(1 / k), 0, trunc_bits=FRAC))
        y = _sub(y, s)
    return y


def max_lastdim(x, seed, ops):
    """Max over the last axis of shares x [P, ..., m] by a tree over adjacent pairs."""
    x = np.asarray(x, dtype=U64)
    P, m = x.shape[0], x.shape[-1]
    vals = x.reshape(P, -1, m)
    while vals.shape[-1] > 1:
        m = vals.shape[-1]
        npairs = m // 2
        a = vals[:, :, 0:2 * npairs:2]
        b = vals[:, :, 1:2 * npairs:2]
        r = relu_shares(np.ascontiguousarray(_sub(a, b)), ops.take(), seed)
        new = _add(b, r)
        if m % 2:
            new = np.concatenate([new, vals[:, :, m - 1:]], axis=2)
        vals = new
    return vals[:, :, 0].reshape(x.shape[:-1])


def softmax(x, seed, ops, recip_iters=10):
    """Softmax over the last axis: exp(x - max) * reciprocal(sum exp(x - max))."""
    x = np.asarray(x, dtype=U64)
    mx = max_lastdim(x, seed, ops)
    e = exp(_sub(x, mx[..., None]), seed, ops)
    with np.errstate(over="ignore"):
        s = e.sum(axis=-1, dtype=U64)
    r = reciprocal_pos(s, seed, ops, recip_iters)
    rb = np.ascontiguousarray(np.broadcast_to(r[..., None], e.shape))
    return mul(e, rb, seed, ops)
