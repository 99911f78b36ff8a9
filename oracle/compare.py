"""Comparators and multiplexing from [z < 0] (§5.2, App. D.1.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

With ltz(z) = [z < 0] (an unscaled 0/1 sharing):
    [x < y] = ltz(x - y)          [x > y] = ltz(y - x)
    [x >= y] = 1 - [x < y]        [x <= y] = 1 - [x > y]
    [x == y] = [x <= y] - [x < y] [x != y] = 1 - [x == y]
and multiplexing [c ? x : y] = [c]([x] - [y]) + [y] (a Beaver product with
the unscaled bit, no truncation).  Public 1 is added by party 0.  Each ltz
consumes its own dealer material (AND triples, B2A pair) and A2B masks,
drawn at op, op+1 and op+3 (the same op-id convention as ReLU).
"""
import numpy as np

from . import beaver, binary, dealer
from .beaver import affine

U64 = np.uint64


def _ltz_material(z, seed, op):
    P, n = z.shape
    T = dealer.and_triples(P, n, binary.KS_GATES * (P - 1), seed, op)
    ra, rb = dealer.b2a_bits(P, n, seed, op + 1)
    return T, ra, rb


def ltz(z, seed, op, tr=None):
    T, ra, rb = _ltz_material(z, seed, op)
    return binary.ltz(z, T, ra, rb, seed, op + 3, tr)


def _sub(x, y):
    with np.errstate(over="ignore"):
        return np.asarray(x, dtype=U64) - np.asarray(y, dtype=U64)


def lt(x, y, seed, op, tr=None):
    return ltz(_sub(x, y), seed, op, tr)


def gt(x, y, seed, op, tr=None):
    return ltz(_sub(y, x), seed, op, tr)


def ge(x, y, seed, op, tr=None):
    return affine(lt(x, y, seed, op, tr), -1, 1)


def le(x, y, seed, op, tr=None):
    return affine(gt(x, y, seed, op, tr), -1, 1)


def eq(x, y, seed, op, tr=None):
    """[x <= y] - [x < y]; the two comparisons use op and op + 10."""
    return _sub(le(x, y, seed, op, tr), lt(x, y, seed, op + 10, tr))


def ne(x, y, seed, op, tr=None):
    return affine(eq(x, y, seed, op, tr), -1, 1)


def mux(c, x, y, seed, op, tr=None):
    """[c ? x : y] with the elementwise triple at op (c an unscaled 0/1 sharing)."""
    c = np.asarray(c, dtype=U64)
    P, n = c.shape
    A, B, C = dealer.mul_triple(P, n, seed, op)
    with np.errstate(over="ignore"):
        return beaver.beaver_mul(c, _sub(x, y), A, B, C, tr) + np.asarray(y, dtype=U64)
