"""Beaver multiplication over arithmetic shares for any bilinear f.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§5.2 "Private multiplication" and App. D.1.1 "Multiplication": with a triple
([a], [b], [c]), c = f(a, b), the parties form [eps] = [x] - [a] and
[delta] = [y] - [b], open eps and delta (one round), and compute
    [f(x, y)] = [c] + f(eps, [b]) + f([a], delta) + f(eps, delta),
where the public term f(eps, delta) is added by one party (party 0 here).
The same identity serves elementwise products, matmul and convolution.
"""
import numpy as np

from . import ring
from .sharing import reveal
from .transcript import _maybe

U64 = np.uint64


def beaver(X, Y, A, B, C, f, tr=None):
    """Generic Beaver product of shares X [P,...], Y [P,...] under bilinear f."""
    tr = _maybe(tr)
    X, Y, A, B, C = (np.asarray(t, dtype=U64) for t in (X, Y, A, B, C))
    P = X.shape[0]
    with np.errstate(over="ignore"):
        eps = reveal(X - A)       # opened
        delta = reveal(Y - B)     # opened (same round as eps)
        tr.open(eps.nbytes)
        tr.open(delta.nbytes)
        tr.next_round()
        Z = []
        for p in range(P):
            z = C[p] + f(eps, B[p]) + f(A[p], delta)
            if p == 0:
                z = z + f(eps, delta)
            Z.append(z)
    return np.stack(Z), eps, delta


def _mul(a, b):
    with np.errstate(over="ignore"):
        return a * b


def beaver_mul(X, Y, A, B, C, tr=None):
    """Elementwise product; returns Z [P][n]."""
    return beaver(X, Y, A, B, C, _mul, tr)[0]


def beaver_matmul(X, Y, A, B, C, tr=None):
    """X [P][M][K], Y [P][K][N] -> Z [P][M][N]."""
    return beaver(X, Y, A, B, C, ring.matmul, tr)[0]


def beaver_conv2d(X, W, A, B, C, stride, pad, pad_w=None, tr=None):
    """X [P][N][Cin][H][W] (data), W [P][Cout][Cin][kh][kw] (weights)."""
    f = lambda x, w: ring.conv2d(x, w, stride=stride, pad=pad, pad_w=pad_w)
    return beaver(X, W, A, B, C, f, tr)[0]


def beaver_square(X, A, B, tr=None):
    """App. D.1.1 "Square": open eps = x - a, [x^2] = [b] + 2 eps [a] + eps^2 (party 0)."""
    tr = _maybe(tr)
    X, A, B = (np.asarray(t, dtype=U64) for t in (X, A, B))
    with np.errstate(over="ignore"):
        eps = reveal(X - A)
        tr.open(eps.nbytes)
        tr.next_round()
        Z = B + U64(2) * eps[None] * A
        Z[0] += eps * eps
    return Z


def affine(X, scale, offset=0, trunc_bits=0):
    """Local: Z_p = scale * X_p (+ offset on party 0), then optional two-party truncation.

    scale is a public integer and offset a public ring element (§5.2: products
    and sums with public values are local).
    """
    from .truncation import truncate
    X = np.asarray(X, dtype=U64)
    with np.errstate(over="ignore"):
        Z = X * U64(int(scale) % (1 << 64))
        Z[0] += U64(int(offset) % (1 << 64))
    return truncate(Z, trunc_bits) if trunc_bits else Z
