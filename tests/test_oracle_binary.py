"""Pins for binary AND, the Kogge-Stone adder, A2B, B2A (Alg. 2), comparator, ReLU.

Expected values are plain integer facts: x & y, (x + y) mod 2^64 by Python
ints, max(s(x), 0), Alg. 2's truth table, and Table 3's round counts.
"""
import itertools

import numpy as np
import pytest

from oracle import binary, dealer, sharing
from oracle.transcript import Transcript

M64 = (1 << 64) - 1


def _bshare(x, P, seed):
    """Binary sharing for tests: P-1 random words, last = x ^ rest."""
    r = np.random.default_rng(seed)
    S = r.integers(0, 2 ** 64, (P, x.size), dtype=np.uint64)
    S[P - 1] = x ^ sharing.reveal_xor(S[:P - 1]) if P > 1 else x
    return S


@pytest.mark.parametrize("P", [2, 3, 4])
def test_and_gate(P, rng):
    x = rng.integers(0, 2 ** 64, 500, dtype=np.uint64)
    y = rng.integers(0, 2 ** 64, 500, dtype=np.uint64)
    T = dealer.and_triples(P, 500, 1, 1, 1)
    tr = Transcript()
    z = binary.and_gate(_bshare(x, P, 1), _bshare(y, P, 2), T[0, 0], T[0, 1], T[0, 2], tr)
    assert np.array_equal(sharing.reveal_xor(z), x & y)
    assert tr.rounds == 1


def test_and_triples_are_ands():
    T = dealer.and_triples(3, 64, 12, 1, 9)
    for g in range(12):
        a, b, c = (sharing.reveal_xor(T[g, i]) for i in range(3))
        assert np.array_equal(c, a & b)


def _ks(x, y, seed=4):
    T = dealer.and_triples(2, x.size, binary.KS_GATES, 1, seed)
    tr = Transcript()
    s = sharing.reveal_xor(binary.ks_add(_bshare(x, 2, 5), _bshare(y, 2, 6), T, tr))
    return s, tr


def test_ks_adder_exhaustive_bytes():
    """All 2^16 pairs of 8-bit addends, including the carry out of bit 7."""
    a, b = np.meshgrid(np.arange(256, dtype=np.uint64), np.arange(256, dtype=np.uint64))
    x, y = a.reshape(-1), b.reshape(-1)
    s, _ = _ks(x, y)
    assert np.array_equal(s, x + y)
    # The same pairs placed in the top byte: carries fall off the ring.
    s2, _ = _ks(x << np.uint64(56), y << np.uint64(56))
    with np.errstate(over="ignore"):
        assert np.array_equal(s2, (x << np.uint64(56)) + (y << np.uint64(56)))


def test_ks_adder_random_and_carry_chains(rng):
    pats = [(M64, 1), (M64, M64), (0x5555555555555555, 0xAAAAAAAAAAAAAAAB),
            (1 << 63, 1 << 63), (0x7FFFFFFFFFFFFFFF, 1), (0, 0), (0xFFFFFFFF, 1)]
    x = np.array([p[0] for p in pats] + [int(v) for v in rng.integers(0, 2 ** 64, 2000, dtype=np.uint64)],
                 dtype=np.uint64)
    y = np.array([p[1] for p in pats] + [int(v) for v in rng.integers(0, 2 ** 64, 2000, dtype=np.uint64)],
                 dtype=np.uint64)
    s, tr = _ks(x, y)
    assert [int(v) for v in s] == [(int(a) + int(b)) & M64 for a, b in zip(x, y)]
    assert tr.rounds == 7     # 1 generate round + log2(64) prefix rounds


def test_a2b_reconstructs_the_secret(rng):
    x = rng.integers(0, 2 ** 64, 3000, dtype=np.uint64)
    x[:4] = [0, M64, 1 << 63, 1]
    X = sharing.share(x, 2, 0, 3, 3)
    T = dealer.and_triples(2, x.size, 12, 3, 4)
    tr = Transcript()
    b = binary.a2b(X, T, 3, 5, tr)
    assert np.array_equal(sharing.reveal_xor(b), x)
    assert tr.rounds == 7     # Table 3: log2|P| * log2(bits) = 1 * 6, +1 generate


def test_a2b_one_party_is_the_identity():
    """A tree of ceil(log2 1) = 0 adder levels: the binary sharing of the one
    share is the share itself, with no AND gate and no round."""
    x = np.array([[0, 1, M64, 1 << 63, 12345]], dtype=np.uint64)
    tr = Transcript()
    assert np.array_equal(binary.a2b(x, np.zeros((0, 3, 1, 5), dtype=np.uint64), 1, 1, tr), x)
    assert tr.rounds == 0
    with pytest.raises(ValueError):
        binary.a2b(np.zeros((0, 4), dtype=np.uint64), None, 1, 1)


@pytest.mark.parametrize("P,levels", [(3, 2), (4, 2), (5, 3), (8, 3)])
def test_a2b_adder_tree(P, levels, rng):
    """|P| > 2: a tree of adders; 7 rounds per level (Table 3: log2|P| log2 L)."""
    x = rng.integers(0, 2 ** 64, 1500, dtype=np.uint64)
    x[:3] = [0, M64, 1 << 63]
    X = sharing.share(x, P, P - 1, 3, 3)
    T = dealer.and_triples(P, x.size, 12 * (P - 1), 3, 4)
    tr = Transcript()
    b = binary.a2b(X, T, 3, 5, tr)
    assert np.array_equal(sharing.reveal_xor(b), x)
    # adders of one level run in parallel, so the rounds count levels
    assert tr.rounds == 7 * (P - 1)   # this oracle evaluates adders one after another


def test_b2a_truth_table():
    """Alg. 2 over every (b, r) and every split of both into two binary shares."""
    rows = []
    for b, r, b0, r0 in itertools.product([0, 1], repeat=4):
        rows.append((b, r, b0, b ^ b0, r0, r ^ r0))
    rows = np.array(rows, dtype=np.uint64)
    n = rows.shape[0]
    b, r = rows[:, 0], rows[:, 1]
    bits = np.stack([rows[:, 2], rows[:, 3]])
    r_bin = np.stack([rows[:, 4], rows[:, 5]])
    ra0 = np.random.default_rng(0).integers(0, 2 ** 64, n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        r_arith = np.stack([ra0, r - ra0])
    tr = Transcript()
    out = binary.b2a_bit(bits, r_arith, r_bin, tr)
    assert np.array_equal(sharing.reveal(out), b)
    assert tr.rounds == 1


@pytest.mark.parametrize("P", [2, 3, 5])
def test_b2a_pairs_share_one_bit(P):
    ra, rb = dealer.b2a_bits(P, 4000, 1, 77)
    r = dealer.secret_bit(4000, 1, 77)
    assert np.array_equal(sharing.reveal(ra), r)
    assert np.array_equal(sharing.reveal_xor(rb), r)
    assert set(np.unique(rb).tolist()) <= {0, 1}
    assert 1800 < int(r.sum()) < 2200


EDGE_SIGNED = [0, 1, -1, 2, -2, (1 << 62), -(1 << 62), (1 << 63) - 1, 65536, -65536]


def _relu_material(n, P=2, base=100):
    T = dealer.and_triples(P, n, 12, 1, base)
    ra, rb = dealer.b2a_bits(P, n, 1, base + 1)
    mt = dealer.mul_triple(P, n, 1, base + 2)
    return T, ra, rb, mt


def test_gt_zero(rng):
    v = np.array(EDGE_SIGNED + [int(t) for t in rng.integers(-(1 << 50), 1 << 50, 2000)], dtype=np.int64)
    X = sharing.share(v.view(np.uint64), 2, 0, 1, 1)
    T, ra, rb, _ = _relu_material(v.size)
    got = sharing.reveal(binary.gt_zero(X, T, ra, rb, 1, 50))
    assert got.tolist() == [1 if t > 0 else 0 for t in v]


def test_gt_zero_most_negative_edge():
    """-2^63 is its own negation: MSB(-x) = 1, so it compares as 'positive'."""
    v = np.array([-(1 << 63)], dtype=np.int64)
    X = sharing.share(v.view(np.uint64), 2, 0, 1, 1)
    T, ra, rb, _ = _relu_material(1)
    assert int(sharing.reveal(binary.gt_zero(X, T, ra, rb, 1, 50))[0]) == 1


def test_private_relu_exact(rng):
    v = np.array(EDGE_SIGNED + [int(t) for t in rng.integers(-(1 << 40), 1 << 40, 3000)], dtype=np.int64)
    X = sharing.share(v.view(np.uint64), 2, 0, 1, 1)
    T, ra, rb, mt = _relu_material(v.size)
    tr = Transcript()
    Y = binary.private_relu(X, T, ra, rb, mt, 1, 51, tr)
    got = sharing.reveal(Y).view(np.int64)
    assert got.tolist() == [max(int(t), 0) for t in v]
    assert tr.rounds == 7 + 1 + 1     # A2B, B2A, Beaver multiply
