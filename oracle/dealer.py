"""Trusted-third-party (TTP) dealer: Beaver triples, AND triples, B2A bit pairs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§4 (the TTP supplies offline material) and App. D.1.1 "Multiplication": a
Beaver triple ([a], [b], [c]) with c = f(a, b) and a, b uniform over the ring.
App. D.1.2 "Bitwise AND": binary triples (<a>, <b>, <c>) with c = a AND b.
App. D.1.3 "From <x> to [x]": pairs ([r], <r>) sharing the same random bit r.

Readings (the paper leaves them open):
  * every party's shares of a and b are fresh PRG words; a = sum_p A_p,
    b = sum_p B_p (XOR for binary);
  * c is shared by drawing C_p for p < P-1 from the PRG and giving the last
    party the correction C_{P-1} = c - sum_{p<P-1} C_p (XOR for binary);
  * the secret bit r of a B2A pair is bit 0 of the TTP's own stream
    (party = TTP_PARTY); <r>_p (bit 0) and [r]_p for p < P-1 are PRG words, and
    the last party gets the corrections.
Word index of every stream = flat (C-order) element index.
"""
import numpy as np

from . import prg, ring
from .sharing import reveal, reveal_xor

U64 = np.uint64


def _streams(P, role, sub, n, seed, op_id):
    return np.stack([prg.stream(seed, op_id, role, sub, p, n) for p in range(P)])


def _share_product(c, P, role_c, sub, seed, op_id):
    """C_p from the PRG for p < P-1, last = c - sum (mod 2^64)."""
    c = np.asarray(c, dtype=U64).reshape(-1)
    C = np.zeros((P, c.size), dtype=U64)
    with np.errstate(over="ignore"):
        acc = np.zeros_like(c)
        for p in range(P - 1):
            C[p] = prg.stream(seed, op_id, role_c, sub, p, c.size)
            acc += C[p]
        C[P - 1] = c - acc
    return C


def mul_triple(P, n, seed, op_id):
    """Elementwise triple: returns A, B, C each [P][n], c = a * b."""
    A = _streams(P, prg.TRIPLE_A, 0, n, seed, op_id)
    B = _streams(P, prg.TRIPLE_B, 0, n, seed, op_id)
    with np.errstate(over="ignore"):
        c = reveal(A) * reveal(B)
    return A, B, _share_product(c, P, prg.TRIPLE_C, 0, seed, op_id)


def matmul_triple(P, M, N, K, seed, op_id):
    """Matmul triple: A [P][M][K], B [P][K][N], C [P][M][N], c = a @ b."""
    A = _streams(P, prg.TRIPLE_A, 0, M * K, seed, op_id).reshape(P, M, K)
    B = _streams(P, prg.TRIPLE_B, 0, K * N, seed, op_id).reshape(P, K, N)
    c = ring.matmul(reveal(A), reveal(B))
    C = _share_product(c, P, prg.TRIPLE_C, 0, seed, op_id).reshape(P, M, N)
    return A, B, C


def conv2d_triple(P, x_shape, w_shape, stride, pad, seed, op_id, pad_w=None):
    """Conv triple: A input-shaped, B weight-shaped, c = conv2d(a, b)."""
    nx = int(np.prod(x_shape))
    nw = int(np.prod(w_shape))
    A = _streams(P, prg.TRIPLE_A, 0, nx, seed, op_id).reshape((P,) + tuple(x_shape))
    B = _streams(P, prg.TRIPLE_B, 0, nw, seed, op_id).reshape((P,) + tuple(w_shape))
    c = ring.conv2d(reveal(A), reveal(B), stride=stride, pad=pad, pad_w=pad_w)
    C = _share_product(c, P, prg.TRIPLE_C, 0, seed, op_id).reshape((P,) + c.shape)
    return A, B, C


def and_triples(P, n, gates, seed, op_id):
    """Binary AND triples for ``gates`` gates: array [gates][3][P][n] (a, b, c)."""
    T = np.zeros((gates, 3, P, n), dtype=U64)
    for g in range(gates):
        A = _streams(P, prg.AND_A, g, n, seed, op_id)
        B = _streams(P, prg.AND_B, g, n, seed, op_id)
        c = reveal_xor(A) & reveal_xor(B)
        C = np.zeros((P, n), dtype=U64)
        acc = np.zeros(n, dtype=U64)
        for p in range(P - 1):
            C[p] = prg.stream(seed, op_id, prg.AND_C, g, p, n)
            acc ^= C[p]
        C[P - 1] = c ^ acc
        T[g, 0], T[g, 1], T[g, 2] = A, B, C
    return T


def b2a_bits(P, n, seed, op_id):
    """Random-bit pairs ([r], <r>) for B2A.

    Returns (r_arith [P][n] uint64, r_bin [P][n] uint64 in {0, 1}).
    """
    one = U64(1)
    r = prg.stream(seed, op_id, prg.B2A_R, 0, prg.TTP_PARTY, n) & one
    r_bin = np.zeros((P, n), dtype=U64)
    r_arith = np.zeros((P, n), dtype=U64)
    accb = np.zeros(n, dtype=U64)
    acca = np.zeros(n, dtype=U64)
    with np.errstate(over="ignore"):
        for p in range(P - 1):
            r_bin[p] = prg.stream(seed, op_id, prg.B2A_BIN, 0, p, n) & one
            r_arith[p] = prg.stream(seed, op_id, prg.B2A_ARITH, 0, p, n)
            accb ^= r_bin[p]
            acca += r_arith[p]
        r_bin[P - 1] = r ^ accb
        r_arith[P - 1] = r - acca
    return r_arith, r_bin


def secret_bit(n, seed, op_id):
    """The TTP's bit r itself (for tests of the pair's consistency)."""
    return prg.stream(seed, op_id, prg.B2A_R, 0, prg.TTP_PARTY, n) & U64(1)


def trunc_pairs(P, n, seed, op_id):
    """Alg. 1 material: [r] uniform (TRUNC_R, sub 0) and shares of theta_r.

    theta_r = (sum_p s(r_p) - s(r)) / Q is the wrap count of r's shares (signed
    view); its shares are TRUNC_R words (sub 1) for p < P-1 and the correction
    on party P-1.  Returns (r [P][n], theta_r [P][n]).
    """
    from .truncation import wrap_count
    R = np.stack([prg.stream(seed, op_id, prg.TRUNC_R, 0, p, n) for p in range(P)])
    th = np.array([wrap_count(R[:, i]) for i in range(n)], dtype=np.int64).view(U64)
    TH = np.zeros((P, n), dtype=U64)
    acc = np.zeros(n, dtype=U64)
    with np.errstate(over="ignore"):
        for p in range(P - 1):
            TH[p] = prg.stream(seed, op_id, prg.TRUNC_R, 1, p, n)
            acc += TH[p]
        TH[P - 1] = th - acc
    return R, TH


def square_pair(P, n, seed, op_id):
    """Beaver pair ([a], [b]) with b = a^2 (App. D.1.1 "Square").

    A_p = TRIPLE_A words for all p; b's shares are TRIPLE_C words for p < P-1
    and the correction on party P-1.  Returns (A, B) each [P][n].
    """
    A = _streams(P, prg.TRIPLE_A, 0, n, seed, op_id)
    with np.errstate(over="ignore"):
        a = reveal(A)
        b = a * a
    return A, _share_product(b, P, prg.TRIPLE_C, 0, seed, op_id)
