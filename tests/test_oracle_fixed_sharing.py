"""Pins for fixed-point encoding (§5.1) and zero-share sharing / reveal (§5.1)."""
import numpy as np
import pytest

from oracle import fixed, sharing

M64 = (1 << 64) - 1


def test_encode_dyadic_values_exact():
    x = np.array([0.0, 1.0, -1.0, 0.5, -2.25, 3.0 / 65536, -1.0 / 65536, 12345.75])
    expect = [0, 65536, -65536, 32768, -147456, 3, -1, 12345 * 65536 + 49152]
    assert fixed.signed(fixed.encode(x)).tolist() == expect


def test_encode_matches_python_round_off_ties(rng):
    x = rng.uniform(-1000, 1000, 2000)
    ours = fixed.signed(fixed.encode(x)).tolist()
    # Python's round() is correctly-rounded on the exact float product (ties are
    # measure-zero for these draws).
    assert ours == [round(v * 65536) for v in x]


def test_encode_ties_half_to_even():
    half = 1.0 / (1 << 17)     # exactly half an ulp of 2^-16
    x = np.array([half, 3 * half, -half, -3 * half, 5 * half])
    assert fixed.signed(fixed.encode(x)).tolist() == [0, 2, 0, -2, 2]


@pytest.mark.parametrize("bad", [2.0 ** 47, -2.0 ** 47, np.inf, np.nan])
def test_encode_range_error(bad):
    with pytest.raises(fixed.EncodeRangeError):
        fixed.encode(np.array([0.0, bad]))


def test_encode_largest_in_range():
    v = np.nextafter(2.0 ** 47, 0.0)          # 2^47 - 2^-6, the last double below
    assert int(fixed.signed(fixed.encode(np.array([v, -v])))[0]) == (1 << 63) - (1 << 10)
    assert int(fixed.signed(fixed.encode(np.array([-v])))[0]) == -(1 << 63) + (1 << 10)


def test_decode_inverts_encode_on_grid(rng):
    k = rng.integers(-(1 << 40), 1 << 40, 500)
    x = k / 65536.0
    assert np.array_equal(fixed.decode(fixed.encode(x)), x)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 8])
def test_shares_sum_to_secret(P, rng):
    x = rng.integers(0, 2 ** 64, 1000, dtype=np.uint64)
    for src in {0, P - 1}:
        S = sharing.share(x, P, src, seed=5, op_id=9)
        tot = [sum(int(S[p, i]) for p in range(P)) & M64 for i in range(x.size)]
        assert tot == [int(v) for v in x]


def test_one_party_share_is_the_secret(rng):
    x = rng.integers(0, 2 ** 64, 64, dtype=np.uint64)
    assert np.array_equal(sharing.share(x, 1, 0, 3, 4)[0], x)


def _chi2_bytes(words):
    b = np.asarray(words, dtype=np.uint64).view(np.uint8)
    counts = np.bincount(b, minlength=256)
    e = b.size / 256.0
    return float(((counts - e) ** 2 / e).sum())


def test_each_share_looks_uniform():
    # A constant secret: every single share must still look like uniform noise.
    x = np.full(1 << 14, 12345, dtype=np.uint64)
    S = sharing.share(x, 2, 0, seed=1, op_id=1)
    for p in range(2):
        # chi^2 with 255 dof: mean 255, sd ~22.6; 400 is > 6 sd.
        assert _chi2_bytes(S[p]) < 400
    assert _chi2_bytes(x) > 1e5     # the secret itself is far from uniform


def test_zero_share_sums_to_zero():
    Z = sharing.zero_share(5, 100, 7, 7)
    assert not np.any(sharing.reveal(Z))
