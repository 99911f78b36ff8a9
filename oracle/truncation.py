"""Two-party local truncation of arithmetic shares.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

App. D.1.1 "Truncation": a shared value is divided by a public l by having
each party divide its own share; this is exact unless the shares wrap around
the ring (probability about |x|/Q for two parties), and costs no communication
for |P| = 2 (Table 3, dagger).

Reading: each share is taken in its signed two's-complement view and divided
with floor rounding (an arithmetic right shift for l = 2^f).  The paper states
neither the signedness nor the rounding direction.
"""
import numpy as np

U64 = np.uint64


def truncate(shares, frac_bits=16, divisor=0):
    """Per-share floor(s(share) / l), l = divisor if nonzero else 2^frac_bits."""
    s = np.asarray(shares, dtype=U64).view(np.int64)
    if divisor:
        if divisor < 0:
            raise ValueError("divisor must be positive")
        out = s // np.int64(divisor)
    else:
        out = s >> np.int64(frac_bits)
    return out.astype(np.int64).view(U64)


# ---- n-party truncation (Alg. 1) --------------------------------------------------
# Reading: all quantities use the signed two's-complement view s(.) of ring
# elements, so that for a shared x in [-2^63, 2^63)
#     x = sum_p s(x_p) - theta_x Q,            Q = 2^64,
# with an integer wrap count theta_x.  Alg. 1 computes a sharing of theta_x:
#     [z] = [x] + [r];   beta_p from  s(x_p) + s(r_p) = s(z_p) + beta_p Q;
#     z = reveal([z]);   theta_z = (sum_p s(z_p) - s(z)) / Q;
#     eta from s(x) + s(r) = s(z) + eta Q, set to 0 (the paper's simplification:
#     wrong with probability about |x| / Q);
#     [theta_x] = theta_z + [beta] - [theta_r] - [eta].
# Then x / l = sum_p s(x_p) / l - theta_x Q / l, and each party keeps
#     floor(s(x_p) / l) - [theta_x]_p (Q / l)       (Q / l needs l | 2^64).
Q_INT = 1 << 64


def _s(v):
    v = int(v)
    return v - Q_INT if v >= (1 << 63) else v


def wrap_count(shares):
    """theta for integer shares: (sum_p s(x_p) - s(x)) / Q, x = sum mod Q (Python ints)."""
    tot = sum(_s(v) for v in shares)
    x = _s(tot % Q_INT)
    assert (tot - x) % Q_INT == 0
    return (tot - x) // Q_INT


def truncate_nparty(shares, r, theta_r, frac_bits=16, tr=None):
    """Alg. 1 with eta = 0 on shares [P][n]; r, theta_r: dealer shares [P][n]."""
    from .transcript import _maybe
    tr = _maybe(tr)
    X = np.asarray(shares, dtype=U64)
    R = np.asarray(r, dtype=U64)
    TR = np.asarray(theta_r, dtype=U64)
    P, n = X.shape
    ell = 1 << frac_bits
    q_over_l = Q_INT // ell
    with np.errstate(over="ignore"):
        Z = X + R
    tr.open(Z[0].nbytes)
    tr.next_round()
    out = np.zeros_like(X)
    for i in range(n):
        beta = [(_s(X[p, i]) + _s(R[p, i]) - _s(Z[p, i])) // Q_INT for p in range(P)]
        theta_z = wrap_count([Z[p, i] for p in range(P)])
        for p in range(P):
            th = beta[p] - _s(TR[p, i]) + (theta_z if p == 0 else 0)
            y = (_s(X[p, i]) >> frac_bits) - th * q_over_l
            out[p, i] = y % Q_INT
    return out
