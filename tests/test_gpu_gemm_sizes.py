"""Ring GEMM and 3-party Beaver matmul at the sweep sizes, checked on samples.

M = N = K in {1024, 2048, 4096, 8192}, words uniform over Z/2^64 (seed 0), both
engines, the same launch configuration bench.py's sweep times.  The oracle
computes a 256 x 256 block of outputs (rows and columns drawn with
default_rng(0).choice, all of K) from the same inputs; the GPU block must be
equal word for word.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, host  # noqa: E402

from oracle import prg, ring, sharing  # noqa: E402


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def _inputs(n):
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64)
    b = rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64)
    return a, b


def _sample(n, k=256):
    r = np.random.default_rng(0)
    return np.sort(r.choice(n, k, replace=False)), np.sort(r.choice(n, k, replace=False))


@pytest.mark.parametrize("n", [1024, 2048, 4096, 8192])
@pytest.mark.parametrize("engine", ["plain", "limb"])
def test_ring_gemm_sweep_sizes(mpc, n, engine):
    a, b = _inputs(n)
    algo = mpc.LIMB if engine == "limb" else mpc.PLAIN
    Z = mpc.ring_gemm(dev(a), dev(b), None, algo=algo)
    mpc.sync_status()
    rows, cols = _sample(n)
    got = host(Z[rows][:, cols].contiguous())
    assert np.array_equal(got, ring.matmul(a[rows], b[:, cols]))
    del Z
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [1024, 2048])
def test_three_party_beaver_matmul_sampled(mpc, n):
    """P = 3 Beaver product (each party one two-pair GEMM of K' = 2K) on samples.

    The oracle regenerates the dealer's triple itself from the PRG streams
    (a and b in full, c only on the sampled block), so no expected value comes
    from the device.
    """
    P, seed, op = 3, 1, 70
    rng = np.random.default_rng(1)
    X = rng.integers(0, 2 ** 64, (P, n, n), dtype=np.uint64)
    Y = rng.integers(0, 2 ** 64, (P, n, n), dtype=np.uint64)
    A, B, C = mpc.ttp_matmul_triple(P, n, n, n, seed, op, algo=mpc.LIMB)
    Z = mpc.beaver_matmul(dev(X), dev(Y), A, B, C, algo=mpc.LIMB)
    mpc.sync_status()
    rows, cols = _sample(n)
    oA = np.stack([prg.stream(seed, op, prg.TRIPLE_A, 0, p, n * n).reshape(n, n) for p in range(P)])
    oB = np.stack([prg.stream(seed, op, prg.TRIPLE_B, 0, p, n * n).reshape(n, n) for p in range(P)])
    blk = np.ix_(rows, cols)
    with np.errstate(over="ignore"):
        c_blk = ring.matmul(sharing.reveal(oA)[rows], sharing.reveal(oB)[:, cols])
        oC = [prg.stream(seed, op, prg.TRIPLE_C, 0, p, n * n).reshape(n, n)[blk] for p in range(P - 1)]
        oC.append(c_blk - sum(oC[1:], oC[0]))
        assert np.array_equal(host(A), oA) and np.array_equal(host(B), oB)
        hC = host(C)
        for p in range(P):
            assert np.array_equal(hC[p][blk], oC[p])
        E = sharing.reveal(X[:, rows, :] - oA[:, rows, :])      # rows of the opened E
        F = sharing.reveal(Y[:, :, cols] - oB[:, :, cols])      # columns of the opened F
        got = host(Z)[:, rows][:, :, cols]
        for p in range(P):
            ref = oC[p] + ring.matmul(E, oB[p][:, cols]) + ring.matmul(oA[p][rows], F)
            if p == 0:
                ref = ref + ring.matmul(E, F)
            assert np.array_equal(got[p], ref)
