"""Pins for the oracle's Philox4x64-10 (the protocol's PRG).

Pinned against numpy.random.Philox, an independent third-party implementation of
the same published generator (Salmon et al., SC'11), and against Python's
arbitrary-precision integers for the 128-bit multiply.
"""
import numpy as np
import pytest

from oracle import prg

M64 = (1 << 64) - 1


def _numpy_block(counter, key):
    """numpy's Philox increments its counter before drawing; feed counter - 1."""
    c = [int(v) for v in counter]
    v = (c[0] | (c[1] << 64) | (c[2] << 128) | (c[3] << 192)) - 1
    v %= 1 << 256
    cm1 = np.array([(v >> (64 * i)) & M64 for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=cm1)
    return bg.random_raw(4)


@pytest.mark.parametrize("counter,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (1, 0)),
    ((5, 7, (3 << 32) | (2 << 8) | 1, 0), (1, 0)),
    ((M64, M64, 12345, 99), (0xDEADBEEF, 42)),
    ((123456789, 1 << 63, M64, M64), (M64, M64)),
])
def test_philox_block_matches_numpy(counter, key):
    ours = prg.philox4x64(np.array(counter, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(ours, _numpy_block(counter, key))


def test_philox_random_blocks_match_numpy(rng):
    ctrs = rng.integers(0, 2 ** 64, (64, 4), dtype=np.uint64)
    keys = rng.integers(0, 2 ** 64, (64, 2), dtype=np.uint64)
    ours = prg.philox4x64(ctrs, keys)
    for i in range(64):
        assert np.array_equal(ours[i], _numpy_block(ctrs[i], keys[i]))


def test_mulhilo64_against_python_ints(rng):
    edge = [0, 1, 2, M64, M64 - 1, 1 << 63, (1 << 32) - 1, 1 << 32, 0xD2E7470EE14C6C93]
    a = np.array(edge + [int(v) for v in rng.integers(0, 2 ** 64, 200, dtype=np.uint64)],
                 dtype=np.uint64)
    b = np.array(list(reversed(edge)) + [int(v) for v in rng.integers(0, 2 ** 64, 200, dtype=np.uint64)],
                 dtype=np.uint64)
    hi, lo = prg.mulhilo64(a, b)
    for i in range(a.size):
        p = int(a[i]) * int(b[i])
        assert int(hi[i]) == p >> 64 and int(lo[i]) == p & M64


@pytest.mark.parametrize("op_id,role,sub,party", [(1, 0, 0, 0), (7, 5, 11, 1), (300, 10, 0, 7),
                                                  (2, 8, 0, 255)])
def test_stream_is_consecutive_numpy_blocks(op_id, role, sub, party):
    """Word j of a stream = word j mod 4 of block j // 4 (counter word 0 = block)."""
    n = 37
    ours = prg.stream(99, op_id, role, sub, party, n)
    w2 = (role << 32) | (sub << 8) | party
    # numpy, started one below block 0, walks blocks 0, 1, 2, ... in counter word 0.
    v = (0 | (op_id << 64) | (w2 << 128)) - 1
    c = np.array([(v >> (64 * i)) & M64 for i in range(4)], dtype=np.uint64)
    ref = np.random.Philox(key=np.array([99, 0], dtype=np.uint64), counter=c).random_raw(n)
    assert np.array_equal(ours, ref)


def test_streams_are_distinct():
    a = prg.stream(1, 1, prg.TRIPLE_A, 0, 0, 16)
    b = prg.stream(1, 1, prg.TRIPLE_A, 0, 1, 16)
    c = prg.stream(1, 2, prg.TRIPLE_A, 0, 0, 16)
    d = prg.stream(2, 1, prg.TRIPLE_A, 0, 0, 16)
    assert len({a.tobytes(), b.tobytes(), c.tobytes(), d.tobytes()}) == 4
