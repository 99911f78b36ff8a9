"""Pins for Beaver square, the public affine map, comparators and multiplexing."""
import numpy as np
import pytest

from oracle import beaver, compare, dealer, fixed, sharing
from oracle.transcript import Transcript

M64 = (1 << 64) - 1


@pytest.mark.parametrize("P", [1, 2, 3, 8])
def test_beaver_square_identity(P, rng):
    x = rng.integers(0, 2 ** 64, 500, dtype=np.uint64)
    x[:3] = [0, M64, 1 << 63]
    X = sharing.share(x, P, 0, 1, 1)
    A, B = dealer.square_pair(P, 500, 1, 2)
    a, b = sharing.reveal(A), sharing.reveal(B)
    assert [int(v) for v in b] == [(int(t) * int(t)) & M64 for t in a]
    tr = Transcript()
    z = sharing.reveal(beaver.beaver_square(X, A, B, tr))
    assert [int(v) for v in z] == [(int(t) * int(t)) & M64 for t in x]
    assert tr.rounds == 1


def test_affine_public_scale_and_offset(rng):
    v = rng.integers(-(1 << 40), 1 << 40, 300)
    X = sharing.share(v.astype(np.int64).view(np.uint64), 2, 0, 1, 3)
    got = sharing.reveal(beaver.affine(X, -3, 12345)).view(np.int64)
    assert got.tolist() == [-3 * int(t) + 12345 for t in v]
    half = sharing.reveal(beaver.affine(X, 1, 0, trunc_bits=1)).view(np.int64)
    assert set(np.unique(half - v // 2).tolist()) <= {-1, 0}


def _shared(v, P=2, op=5):
    return sharing.share(np.asarray(v, dtype=np.int64).view(np.uint64), P, 0, 1, op)


@pytest.mark.parametrize("P", [2, 3])
def test_comparators_truth(P, rng):
    a = rng.integers(-50, 50, 400)
    b = rng.integers(-50, 50, 400)
    b[:100] = a[:100]          # plenty of equal pairs
    X, Y = _shared(a * 65536, P, 5), _shared(b * 65536, P, 6)
    cases = {"lt": a < b, "gt": a > b, "ge": a >= b, "le": a <= b, "eq": a == b, "ne": a != b}
    for name, want in cases.items():
        got = sharing.reveal(getattr(compare, name)(X, Y, 1, 1000)).view(np.int64)
        assert got.tolist() == want.astype(int).tolist(), name


def test_mux_selects(rng):
    a = rng.uniform(-5, 5, 300)
    b = rng.uniform(-5, 5, 300)
    c = rng.integers(0, 2, 300)
    X = sharing.share(fixed.encode(a), 2, 0, 1, 7)
    Y = sharing.share(fixed.encode(b), 2, 1, 1, 8)
    Cs = _shared(c, 2, 9)
    got = fixed.decode(sharing.reveal(compare.mux(Cs, X, Y, 1, 2000)))
    assert np.array_equal(got, np.where(c == 1, fixed.decode(fixed.encode(a)),
                                        fixed.decode(fixed.encode(b))))
