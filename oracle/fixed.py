"""Fixed-point encoding into the ring Z/2^64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§5.1 "Arithmetic secret sharing" and App. D.1.1: a real x_R is encoded as
x = round(B * x_R) with B = 2^L (L = 16 by default, §7 / App. A), and decoded
as x / B.  Ring elements are uint64; the signed view is two's complement.

Reading of the paper: "round to the nearest integer" does not say how ties are
broken; we round half to even (numpy ``rint``).  Multiplying by 2^L is exact in
float64, so the rint is the only rounding.  |B * x_R| >= 2^63 (or a non-finite
x_R) does not fit the signed range and is an error.
"""
import numpy as np

DEFAULT_FRAC_BITS = 16


class EncodeRangeError(ValueError):
    pass


def encode(x_real, frac_bits=DEFAULT_FRAC_BITS):
    """float64 array -> uint64 ring elements, x = rint(x_R * 2^L)."""
    x = np.asarray(x_real, dtype=np.float64)
    scaled = x * float(2 ** frac_bits)
    if not np.all(np.isfinite(scaled)) or np.any(np.abs(scaled) >= 2.0 ** 63):
        raise EncodeRangeError("real value outside the encodable range")
    return np.rint(scaled).astype(np.int64).view(np.uint64)


def signed(x_ring):
    """Two's-complement signed view of ring elements."""
    return np.asarray(x_ring, dtype=np.uint64).view(np.int64)


def decode(x_ring, frac_bits=DEFAULT_FRAC_BITS):
    """uint64 ring elements -> float64, x_R = s(x) / 2^L."""
    return signed(x_ring).astype(np.float64) / float(2 ** frac_bits)
