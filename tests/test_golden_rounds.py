"""Round counts against the paper's Table 3 (tests/golden/table3_round_complexity.txt).

The oracle's transcripts are checked on the CPU; the library's own round
counter (mpc_get_stats) is checked on the GPU.  One reading differs from the
printed formula and is asserted as such: A2B for L = 64 costs log2(64) = 6
prefix rounds per adder level plus the generate round G = x AND y, i.e. 7 per
level, where the table prints log2|P| log2 L (6 for two parties).
"""
import math
import os

import numpy as np
import pytest

from oracle import beaver, binary, dealer, sharing, truncation
from oracle.transcript import Transcript

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_round_complexity.txt")
L = 64
GENERATE_ROUND = 1   # the reading: one AND round before the log2(L) prefix rounds


def table3():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            name, value = line.split(None, 1)
            rows[name] = value.strip()
    return rows


def rounds(name, P=2):
    v = table3()[name]
    if v == "log2(P)*log2(L)":
        return int(math.ceil(math.log2(P)) * math.log2(L))
    return int(v)


def test_fixture_has_every_primitive():
    assert set(table3()) == {"addition", "multiplication", "truncation", "truncation_two_party",
                             "xor", "and", "bit_shift", "a2b", "b2a"}


def test_oracle_multiplication_and_truncation():
    tr = Transcript()
    A, B, C = dealer.mul_triple(2, 16, 1, 1)
    Z = beaver.beaver_mul(A, B, A, B, C, tr)
    assert tr.rounds == rounds("multiplication")
    tr = Transcript()
    truncation.truncate(Z, 16)
    assert tr.rounds == rounds("truncation_two_party")
    tr = Transcript()
    X = sharing.share(np.arange(16, dtype=np.uint64), 3, 0, 1, 2)
    R, TH = dealer.trunc_pairs(3, 16, 1, 3)
    truncation.truncate_nparty(X, R, TH, 16, tr)
    assert tr.rounds == rounds("truncation")


def test_oracle_and_a2b_b2a():
    n = 64
    x = np.random.default_rng(0).integers(0, 2 ** 64, n, dtype=np.uint64)
    X = sharing.share(x, 2, 0, 1, 4)
    T = dealer.and_triples(2, n, 12, 1, 5)
    tr = Transcript()
    b = binary.a2b(X, T, 1, 6, tr)
    assert tr.rounds == rounds("a2b") + GENERATE_ROUND
    tr = Transcript()
    binary.and_gate(b, b, T[0][0], T[0][1], T[0][2], tr)
    assert tr.rounds == rounds("and")
    ra, rb = dealer.b2a_bits(2, n, 1, 7)
    tr = Transcript()
    binary.b2a_bit(binary.msb(b), ra, rb, tr)
    assert tr.rounds == rounds("b2a")


@pytest.mark.gpu
def test_library_round_counter():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as mpc
    from gpu_util import dev
    n = 1000
    X = dev(sharing.share(np.arange(n, dtype=np.uint64), 2, 0, 1, 8))

    def counted(fn):
        torch.cuda.synchronize()
        mpc.reset_stats()
        fn()
        torch.cuda.synchronize()
        return mpc.get_stats()["rounds"]

    A, B, C = mpc.ttp_mul_triple(2, n, 1, 9)
    assert counted(lambda: mpc.beaver_mul(X, X, A, B, C)) == rounds("multiplication")
    assert counted(lambda: mpc.truncate(X)) == rounds("truncation_two_party")
    assert counted(lambda: mpc.add(X, X)) == rounds("addition")
    T = mpc.ttp_and_triples(2, n, 1, 10)
    assert counted(lambda: mpc.a2b(X, T, 1, 11)) == rounds("a2b") + GENERATE_ROUND
    # private ReLU: A2B, B2A, one multiplication
    assert counted(lambda: mpc.private_relu_fused(X, 1, 12)) == \
        rounds("a2b") + GENERATE_ROUND + rounds("b2a") + rounds("multiplication")
