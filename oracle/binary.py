"""Binary shares: AND, carry-lookahead adder, A2B, B2A, comparator, ReLU.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Definitions followed:
  * Binary sharing over Z/2 packed in 64-bit words, XOR/shift local
    (§5.1 "Binary secret sharing", App. D.1.2).
  * AND with a binary triple (App. D.1.2 "Bitwise AND"): open
    eps = x ^ a and delta = y ^ b (one round), then
    <z> = <c> ^ (eps & <b>) ^ (<a> & delta) ^ (eps & delta), the public term
    on party 0.
  * A2B (§5.1, App. D.1.3 "From [x] to <x>"): every party binary-shares its
    arithmetic share, and the binary shares are summed with a
    carry-lookahead adder.
  * B2A of one bit (Alg. 2): z = reveal(<b> ^ <r>), [b] = [r] + z - 2 z [r].
  * Comparator [z < 0] = B2A(MSB(A2B([z]))) (§5.2 "Comparators"), with
    [x > 0] = [(0 - x) < 0], and ReLU([x]) = [x] * [x > 0] (§5.2, App. D.1.4).

Readings (the paper is silent or inconsistent):
  * The binary sharing of party q's arithmetic share y_q is the binary analogue
    of the zero-share: party p holds M_{q,p} ^ M_{q,(p-1) mod P} ^ [p = q] y_q
    with M_{q,p} from the ZERO_BIN stream (sub = q).
  * The adder is a Kogge-Stone prefix adder.  Generate G = x & y (one secret
    AND, gate 0), propagate P = x ^ y.  For d = 1, 2, 4, 8, 16, 32 (one round
    each): G <- G ^ (P & (G << d)) (a secret AND), and for d < 32 also
    P <- P & (P << d) (a secret AND, same round).  sum = (x ^ y) ^ (G << 1).
    Gates are numbered g0 = generate, then per d the G-update before the
    P-update: 12 gates, 7 rounds.  G and P & (G << d) are never both 1, so
    XOR stands for OR.
  * "<z> >> (L-1)" in the comparator reads as the most significant bit, bit 63,
    of the 64-bit word.
  * The ReLU's product with the 0/1 mask is not truncated: the mask is an
    unscaled integer.
  * For |P| > 2 the P binary-shared addends are summed by a tree of adders
    (§5.1: log2|P| levels): each level adds neighbours (0, 1), (2, 3), ...
    and passes an odd last addend up unchanged; adders are numbered level by
    level, left to right, and adder a uses AND gates 12a .. 12a + 11.
"""
import numpy as np

from . import prg
from .beaver import beaver_mul
from .sharing import reveal_xor
from .transcript import _maybe

U64 = np.uint64
KS_GATES = 12
KS_DISTANCES = (1, 2, 4, 8, 16, 32)
MSB_SHIFT = U64(63)


def and_gate(x, y, a, b, c, tr=None):
    """Secret AND of binary shares x, y [P][n] with triple (a, b, c) [P][n]."""
    tr = _maybe(tr)
    x, y, a, b, c = (np.asarray(t, dtype=U64) for t in (x, y, a, b, c))
    eps = reveal_xor(x ^ a)
    delta = reveal_xor(y ^ b)
    tr.open(eps.nbytes)
    tr.open(delta.nbytes)
    z = c ^ (eps[None] & b) ^ (a & delta[None])
    z[0] ^= eps & delta
    return z


def ks_add(x, y, and_triples, tr=None):
    """Kogge-Stone sum of binary-shared words x, y [P][n] (mod 2^64).

    and_triples: [KS_GATES][3][P][n] (a, b, c) in gate order.
    """
    tr = _maybe(tr)
    x = np.asarray(x, dtype=U64)
    y = np.asarray(y, dtype=U64)
    T = np.asarray(and_triples, dtype=U64)
    gate = 0

    def AND(u, v):
        nonlocal gate
        out = and_gate(u, v, T[gate, 0], T[gate, 1], T[gate, 2], tr)
        gate += 1
        return out

    G = AND(x, y)
    tr.next_round()
    Pp = x ^ y
    P0 = Pp.copy()
    for d in KS_DISTANCES:
        sh = U64(d)
        G_new = G ^ AND(Pp, G << sh)
        if d < 32:
            Pp = AND(Pp, Pp << sh)
        G = G_new
        tr.next_round()
    assert gate == KS_GATES
    return P0 ^ (G << U64(1))


def binary_share_of_share(arith, q, seed, op_id):
    """<y_q>: binary sharing of party q's arithmetic share, returns [P][n]."""
    arith = np.asarray(arith, dtype=U64)
    P, n = arith.shape
    M = np.stack([prg.stream(seed, op_id, prg.ZERO_BIN, q, p, n) for p in range(P)])
    out = M ^ np.roll(M, 1, axis=0)
    out[q] ^= arith[q]
    return out


def a2b(arith, and_triples, seed, op_id, tr=None):
    """[x] -> <x>; arith [P][n], returns binary shares [P][n].

    and_triples: [12 (P - 1)][3][P][n], twelve gates per adder of the tree.
    The tree has ceil(log2 P) levels; for P = 1 it has none, and the single
    party's binary sharing of its own share (the masks cancel) is the result.
    """
    arith = np.asarray(arith, dtype=U64)
    P = arith.shape[0]
    if P < 1:
        raise ValueError("A2B needs at least one party")
    T = np.asarray(and_triples, dtype=U64) if P > 1 else None
    vals = [binary_share_of_share(arith, q, seed, op_id) for q in range(P)]
    adder = 0
    while len(vals) > 1:
        new = []
        for i in range(0, len(vals) - 1, 2):
            new.append(ks_add(vals[i], vals[i + 1], T[KS_GATES * adder:KS_GATES * (adder + 1)], tr))
            adder += 1
        if len(vals) % 2:
            new.append(vals[-1])
        vals = new
    return vals[0]


def msb(binary):
    """Sign bit of binary shares (local shift)."""
    return np.asarray(binary, dtype=U64) >> MSB_SHIFT


def b2a_bit(bits, r_arith, r_bin, tr=None):
    """Alg. 2: binary-shared bit (values 0/1 per party) -> arithmetic share."""
    tr = _maybe(tr)
    bits = np.asarray(bits, dtype=U64)
    r_arith = np.asarray(r_arith, dtype=U64)
    r_bin = np.asarray(r_bin, dtype=U64)
    z = reveal_xor(bits ^ r_bin)          # opened, one round
    tr.open((z.size + 7) // 8)
    tr.next_round()
    with np.errstate(over="ignore"):
        out = r_arith - U64(2) * z[None] * r_arith
        out[0] += z
    return out


def gt_zero(x, and_triples, r_arith, r_bin, seed, op_id, tr=None):
    """[x > 0] = [(0 - x) < 0] as arithmetic shares of a 0/1 bit."""
    x = np.asarray(x, dtype=U64)
    with np.errstate(over="ignore"):
        neg = U64(0) - x
    b = a2b(neg, and_triples, seed, op_id, tr)
    return b2a_bit(msb(b), r_arith, r_bin, tr)


def private_relu(x, and_triples, r_arith, r_bin, mul_triple, seed, op_id, tr=None):
    """ReLU([x]) = [x] * [x > 0]; mul_triple = (A, B, C) each [2][n]."""
    mask = gt_zero(x, and_triples, r_arith, r_bin, seed, op_id, tr)
    A, B, C = mul_triple
    return beaver_mul(x, mask, A, B, C, tr)


def ltz(x, and_triples, r_arith, r_bin, seed, op_id, tr=None):
    """[x < 0] = B2A(MSB(A2B([x]))) (§5.2 "Comparators"), arithmetic 0/1 shares."""
    b = a2b(np.asarray(x, dtype=U64), and_triples, seed, op_id, tr)
    return b2a_bit(msb(b), r_arith, r_bin, tr)
