"""Philox4x64-10 counter-based PRG and the protocol's randomness streams.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper asks for a "pseudorandom zero-share" and for a trusted third party
(TTP) that hands out random triples and bits (§5.1 "Arithmetic secret sharing",
§4 TTP, App. D.1.1 "Multiplication"), but never names a generator.  This module
fixes one so that two independent implementations can agree bit for bit:
Philox4x64 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11).

Philox4x64 round (published definition):
    (hi0, lo0) = mulhilo64(M0, c0);  (hi1, lo1) = mulhilo64(M1, c2)
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
and between consecutive rounds the key is bumped by the Weyl constants:
    k0 += W0, k1 += W1   (mod 2^64).
M0, M1 are the published Philox4x64 multipliers, W0 is the golden-ratio and
W1 the sqrt(3)-1 Weyl increments.

Stream convention (our specification; the paper is silent):
    key     = (seed, 0)
    counter = (block, op_id, (role << 32) | (sub << 8) | party, 0)
    word j of stream (seed, op_id, role, sub, party) is output word (j mod 4)
    of block floor(j / 4).
"""
import numpy as np

U64 = np.uint64
MASK32 = U64(0xFFFFFFFF)

PHILOX_M0 = U64(0xD2E7470EE14C6C93)
PHILOX_M1 = U64(0xCA5A826395121157)
PHILOX_W0 = U64(0x9E3779B97F4A7C15)
PHILOX_W1 = U64(0xBB67AE8584CAA73B)
PHILOX_ROUNDS = 10

# Stream roles.
ZERO_ARITH = 0   # arithmetic pseudorandom zero-share, sub = 0
ZERO_BIN = 1     # binary zero-share used by A2B, sub = owner q of the share
TRIPLE_A = 2     # Beaver triple operand a (elementwise, matmul, conv)
TRIPLE_B = 3     # Beaver triple operand b
TRIPLE_C = 4     # Beaver triple product shares c_p, p < P-1
AND_A = 5        # binary AND triple a, sub = gate index
AND_B = 6        # binary AND triple b
AND_C = 7        # binary AND triple c shares
B2A_R = 8        # the TTP's secret random bit r (party = TTP_PARTY)
B2A_BIN = 9      # binary shares <r>_p, p < P-1
B2A_ARITH = 10   # arithmetic shares [r]_p, p < P-1
TRUNC_R = 11     # n-party truncation mask (reserved)

TTP_PARTY = 255


def mulhilo64(a, b):
    """Full 64x64 -> 128-bit product of uint64 arrays, as (hi, lo).

    Schoolbook multiplication on 32-bit halves; every partial product fits in
    64 bits, so numpy's uint64 arithmetic is exact here.
    """
    a = np.asarray(a, dtype=U64)
    b = np.asarray(b, dtype=U64)
    a0, a1 = a & MASK32, a >> U64(32)
    b0, b1 = b & MASK32, b >> U64(32)
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> U64(32)) + (p01 & MASK32) + (p10 & MASK32)
    lo = (p00 & MASK32) | (mid << U64(32))
    hi = p11 + (p01 >> U64(32)) + (p10 >> U64(32)) + (mid >> U64(32))
    return hi, lo


def philox4x64(counter, key, rounds=PHILOX_ROUNDS):
    """Philox4x64-R bijection.

    counter: uint64 array of shape (..., 4); key: uint64 array of shape (..., 2)
    (broadcastable).  Returns uint64 array of shape (..., 4).
    """
    c = np.asarray(counter, dtype=U64)
    k = np.asarray(key, dtype=U64)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    with np.errstate(over="ignore"):
        for r in range(rounds):
            if r > 0:
                k0 = k0 + PHILOX_W0
                k1 = k1 + PHILOX_W1
            hi0, lo0 = mulhilo64(PHILOX_M0, c0)
            hi1, lo1 = mulhilo64(PHILOX_M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return np.stack(np.broadcast_arrays(c0, c1, c2, c3), axis=-1)


def stream_word2(role, sub, party):
    """Third counter word: (role << 32) | (sub << 8) | party."""
    assert 0 <= party < 256 and 0 <= sub < (1 << 24) and 0 <= role < (1 << 32)
    return (int(role) << 32) | (int(sub) << 8) | int(party)


def stream(seed, op_id, role, sub, party, n):
    """First n words of the stream (seed, op_id, role, sub, party)."""
    n = int(n)
    nblocks = (n + 3) // 4
    ctr = np.zeros((nblocks, 4), dtype=U64)
    ctr[:, 0] = np.arange(nblocks, dtype=U64)
    ctr[:, 1] = U64(op_id)
    ctr[:, 2] = U64(stream_word2(role, sub, party))
    key = np.array([seed, 0], dtype=U64)
    return philox4x64(ctr, key).reshape(-1)[:n].copy()
