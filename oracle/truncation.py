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
