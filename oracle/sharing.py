"""Arithmetic secret sharing by a pseudorandom zero-share, and reveal.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§5.1 "Arithmetic secret sharing" / App. D.1.1: the parties draw a pseudorandom
zero-share (|P| numbers summing to 0 mod Q), and the party owning x adds x to its
share.  Reveal sums all shares mod Q = 2^64.

Zero-share construction (our reading; the paper cites Cramer et al. without
fixing one): R_p is party p's PRG stream (role ZERO_ARITH) and
    share_p = R_p - R_{(p-1) mod P} + [p = src] * x,
which telescopes to x when summed over p.
"""
import numpy as np

from . import prg

U64 = np.uint64


def zero_share(P, n, seed, op_id):
    """[P][n] uint64 shares of zero."""
    R = np.stack([prg.stream(seed, op_id, prg.ZERO_ARITH, 0, p, n) for p in range(P)])
    with np.errstate(over="ignore"):
        return R - np.roll(R, 1, axis=0)


def share(x_ring, P, src, seed, op_id):
    """Share ring elements x (any shape) among P parties; returns [P, *shape]."""
    x = np.asarray(x_ring, dtype=U64)
    if not (1 <= P <= 255) or not (0 <= src < P):
        raise ValueError("bad party count or source party")
    z = zero_share(P, x.size, seed, op_id)
    with np.errstate(over="ignore"):
        z[src] += x.reshape(-1)
    return z.reshape((P,) + x.shape)


def reveal(shares):
    """Sum of shares over the party axis (axis 0), mod 2^64."""
    s = np.asarray(shares, dtype=U64)
    out = np.zeros(s.shape[1:], dtype=U64)
    with np.errstate(over="ignore"):
        for p in range(s.shape[0]):
            out += s[p]
    return out


def reveal_xor(shares):
    """XOR of binary shares over the party axis."""
    s = np.asarray(shares, dtype=U64)
    out = np.zeros(s.shape[1:], dtype=U64)
    for p in range(s.shape[0]):
        out ^= s[p]
    return out
