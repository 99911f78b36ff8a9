"""Parity of the tcgen05 limb-split ring GEMM engine against the oracle, bit-exact.

The limb engine cuts each word into 8 balanced base-256 digits held exactly in
bf16, accumulates the 36 digit pairs with i + j < 8 in fp32 tensor memory and
drains shift s every 1024 / (s + 1) K-steps so no partial sum leaves the range
where fp32 is exact.  The adversarial cases below drive every digit to -128,
so each full chunk sums to exactly 2^24, the edge of exactness.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, host  # noqa: E402

from oracle import beaver, dealer, ring, truncation  # noqa: E402

M64 = (1 << 64) - 1
SEED = 1
ALL_MINUS_128 = 0x7F7F7F7F7F7F7F80   # balanced digits all equal to -128
ALL_PLUS_127 = 0x7F7F7F7F7F7F7F7F


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def u64(rng, shape):
    a = rng.integers(0, 2 ** 64, shape, dtype=np.uint64)
    flat = a.reshape(-1)
    edge = [0, 1, M64, 1 << 63, (1 << 63) - 1, ALL_MINUS_128, ALL_PLUS_127]
    flat[: min(len(edge), flat.size)] = edge[: flat.size]
    return a


def _gemm_ref(a, b, c=None):
    with np.errstate(over="ignore"):
        z = ring.matmul(a, b)
        return z + c if c is not None else z


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (128, 64, 16), (7, 9, 3), (129, 65, 17),
                                   (256, 128, 128), (200, 300, 129), (130, 70, 1000)])
def test_ring_gemm_limb_random(mpc, M, N, K, rng):
    a, b, c = u64(rng, (M, K)), u64(rng, (K, N)), u64(rng, (M, N))
    Z = mpc.ring_gemm(dev(a), dev(b), dev(c), algo=mpc.LIMB)
    mpc.sync_status()
    assert np.array_equal(host(Z), _gemm_ref(a, b, c))


@pytest.mark.parametrize("K", [128, 1024, 2048 + 48])
def test_ring_gemm_limb_exactness_edge(mpc, K):
    """Every digit -128: each shift-7 chunk of 128 K-steps sums 8 x 128 x 2^14 = 2^24."""
    M, N = 128, 64
    a = np.full((M, K), ALL_MINUS_128, dtype=np.uint64)
    b = np.full((K, N), ALL_MINUS_128, dtype=np.uint64)
    Z = mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.LIMB)
    mpc.sync_status()
    assert np.array_equal(host(Z), _gemm_ref(a, b))
    a2 = np.full((M, K), M64, dtype=np.uint64)
    Z2 = mpc.ring_gemm(dev(a2), dev(b), None, algo=mpc.LIMB)
    assert np.array_equal(host(Z2), _gemm_ref(a2, b))


def test_ring_gemm_limb_exactness_full_chunks(mpc, rng):
    """148 tiles and K = 2096 run unsplit, so every shift s reaches a full chunk of
    64 / (s + 1) sub-steps of K = 16; with all digits -128 each sums to 2^24.
    Constant rows of A make every entry a closed form: Z[i, j] = a * sum_k B[k, j]."""
    M, N, K = 512, 37 * 128, 2096
    a = np.full((M, K), ALL_MINUS_128, dtype=np.uint64)
    b = np.full((K, N), ALL_MINUS_128, dtype=np.uint64)
    Z = host(mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.LIMB))
    mpc.sync_status()
    assert np.all(Z == np.uint64(K * ALL_MINUS_128 * ALL_MINUS_128 & M64))
    b = u64(rng, (K, N))
    b[:, :7] = ALL_MINUS_128
    Z = host(mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.LIMB))
    with np.errstate(over="ignore"):
        col = b.sum(axis=0, dtype=np.uint64) * np.uint64(ALL_MINUS_128)
    assert np.array_equal(Z, np.broadcast_to(col, (M, N)))


def test_ring_gemm_limb_mixed_extremes(mpc, rng):
    M, N, K = 192, 192, 640
    choices = np.array([ALL_MINUS_128, ALL_PLUS_127, M64, 0, 1 << 63], dtype=np.uint64)
    a = choices[rng.integers(0, 5, (M, K))]
    b = choices[rng.integers(0, 5, (K, N))]
    Z = mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.LIMB)
    assert np.array_equal(host(Z), _gemm_ref(a, b))


@pytest.mark.parametrize("P,M,N,K,trunc", [(2, 64, 32, 128, 16), (3, 65, 33, 130, 0),
                                           (2, 300, 200, 257, 16), (1, 40, 40, 40, 0)])
def test_beaver_matmul_limb(mpc, P, M, N, K, trunc, rng):
    X, Y = u64(rng, (P, M, K)), u64(rng, (P, K, N))
    A, B, C = dealer.matmul_triple(P, M, N, K, SEED, 61)
    Z = mpc.beaver_matmul(dev(X), dev(Y), dev(A), dev(B), dev(C), algo=mpc.LIMB, trunc_bits=trunc)
    ref = beaver.beaver_matmul(X, Y, A, B, C)
    if trunc:
        ref = truncation.truncate(ref, trunc)
    assert np.array_equal(host(Z), ref)


@pytest.mark.parametrize("P", [2, 3])
def test_matmul_triple_limb(mpc, P):
    M, N, K = 130, 70, 200
    A, B, C = mpc.ttp_matmul_triple(P, M, N, K, SEED, 62, algo=mpc.LIMB)
    rA, rB, rC = dealer.matmul_triple(P, M, N, K, SEED, 62)
    assert np.array_equal(host(C), rC)


@pytest.mark.parametrize("P", [2, 3])
@pytest.mark.parametrize("geom", [
    dict(batch=2, c_in=3, h=9, w=7, c_out=5, k=3, stride=2, pad=1),
    dict(batch=1, c_in=16, h=12, w=12, c_out=130, k=3, stride=1, pad=1),
    # batch 2, stride 2, padding, a non-square input and ragged tiles
    dict(batch=2, c_in=32, h=9, w=11, c_out=24, k=3, stride=2, pad=1),
    # one tap, stride 2 (a ResNet downsampling shortcut)
    dict(batch=2, c_in=16, h=7, w=9, c_out=24, k=1, stride=2, pad=0),
])
def test_beaver_conv2d_limb(mpc, geom, P, rng):
    g = geom
    d = mpc.conv_desc(g["batch"], g["c_in"], g["h"], g["w"], g["c_out"], g["k"], g["k"],
                      g["stride"], g["stride"], g["pad"], g["pad"])
    xs = (g["batch"], g["c_in"], g["h"], g["w"])
    ws = (g["c_out"], g["c_in"], g["k"], g["k"])
    X, W = u64(rng, (P,) + xs), u64(rng, (P,) + ws)
    A, B, C = dealer.conv2d_triple(P, xs, ws, g["stride"], g["pad"], SEED, 63)
    Z = mpc.beaver_conv2d(dev(X), dev(W), dev(A), dev(B), dev(C), d, algo=mpc.LIMB, trunc_bits=16)
    ref = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, g["stride"], g["pad"]), 16)
    assert np.array_equal(host(Z), ref)
    gA, gB, gC = mpc.ttp_conv2d_triple(P, d, SEED, 63, algo=mpc.LIMB)
    assert np.array_equal(host(gC), C)


@pytest.mark.parametrize("P", [2, 3])
@pytest.mark.parametrize("engine", ["limb", "plain"])
@pytest.mark.parametrize("geom", [
    # (batch, c_in, h, w, c_out, kh, kw, stride, pad_h, pad_w)
    (2, 16, 9, 11, 24, 3, 3, 2, 1, 1),     # ragged tiles, one split
    (1, 160, 1, 100, 40, 1, 7, 1, 0, 3),   # K = 1120: the batched GEMM is split along K
])
def test_conv_triples_batch_matches_oracle(mpc, P, engine, geom):
    """A batch of same-shaped convolution triples (one GEMM launch for all their
    products on the limb engine) equals the oracle's triples at each op id."""
    b, ci, h, w, co, kh, kw, st, ph, pw = geom
    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    ops = [70, 81, 92]
    algo = mpc.LIMB if engine == "limb" else mpc.PLAIN
    outs = mpc.ttp_conv2d_triples(P, d, SEED, ops, algo=algo)
    mpc.sync_status()
    for op, (gA, gB, gC) in zip(ops, outs):
        rA, rB, rC = dealer.conv2d_triple(P, (b, ci, h, w), (co, ci, kh, kw), st, ph, SEED, op,
                                          pad_w=pw)
        assert np.array_equal(host(gA), rA)
        assert np.array_equal(host(gB), rB)
        assert np.array_equal(host(gC), rC)


@pytest.mark.parametrize("P", [2, 3])
def test_conv_triples_mixed_descriptors(mpc, P):
    """One batch of triples for convolutions that differ in input channels,
    kernel, stride and padding but share the output shape (c_out 40, 64
    columns): each product has its own K (one GEMM launch, one plane launch per
    run of equal descriptors), the splits capped by the shortest K (a 1 x 1
    convolution of 16 channels: one sub-step)."""
    geoms = [
        # (batch, c_in, h, w, c_out, kh, kw, stride, pad_h, pad_w)
        (1, 160, 1, 64, 40, 1, 7, 1, 0, 3),
        (1, 160, 1, 64, 40, 1, 7, 1, 0, 3),
        (1, 48, 1, 128, 40, 1, 11, 2, 0, 5),
        (1, 16, 1, 64, 40, 1, 1, 1, 0, 0),
    ]
    descs = [mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
             for b, ci, h, w, co, kh, kw, st, ph, pw in geoms]
    ops = [700, 711, 722, 733]
    outs = mpc.ttp_conv2d_triples(P, descs, SEED, ops, algo=mpc.LIMB)
    mpc.sync_status()
    for g, op, (gA, gB, gC) in zip(geoms, ops, outs):
        b, ci, h, w, co, kh, kw, st, ph, pw = g
        rA, rB, rC = dealer.conv2d_triple(P, (b, ci, h, w), (co, ci, kh, kw), st, ph, SEED, op,
                                          pad_w=pw)
        assert np.array_equal(host(gA), rA) and np.array_equal(host(gB), rB)
        assert np.array_equal(host(gC), rC)
    # without the 1 x 1 convolution the batch is split along K
    outs = mpc.ttp_conv2d_triples(P, descs[:3], SEED, ops[:3], algo=mpc.LIMB)
    mpc.sync_status()
    for g, op, (gA, gB, gC) in zip(geoms, ops, outs):
        b, ci, h, w, co, kh, kw, st, ph, pw = g
        _, _, rC = dealer.conv2d_triple(P, (b, ci, h, w), (co, ci, kh, kw), st, ph, SEED, op,
                                        pad_w=pw)
        assert np.array_equal(host(gC), rC)


@pytest.mark.parametrize("P,count", [(8, 2), (2, 8)])
def test_conv_triples_batch_edges(mpc, P, count):
    """Eight parties, and the largest batch, on a tiny convolution (N = 15 output
    columns, M = 8 rows: one ragged tile per product)."""
    b, ci, h, w, co, kh, kw, st, ph, pw = (1, 16, 3, 5, 8, 3, 3, 1, 1, 1)
    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    ops = [300 + 7 * j for j in range(count)]
    outs = mpc.ttp_conv2d_triples(P, d, SEED, ops, algo=mpc.LIMB)
    mpc.sync_status()
    for op, (gA, gB, gC) in zip(ops, outs):
        rA, rB, rC = dealer.conv2d_triple(P, (b, ci, h, w), (co, ci, kh, kw), st, ph, SEED, op,
                                          pad_w=pw)
        assert np.array_equal(host(gA), rA) and np.array_equal(host(gB), rB)
        assert np.array_equal(host(gC), rC)


def test_limb_large_subset(mpc, rng):
    """A 1024^3 product checked on a 64 x 64 sample of outputs with full K."""
    n = 1024
    a, b = u64(rng, (n, n)), u64(rng, (n, n))
    Z = host(mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.LIMB))
    rows = np.sort(rng.choice(n, 64, replace=False))
    cols = np.sort(rng.choice(n, 64, replace=False))
    ref = ring.matmul(a[rows], b[:, cols])
    assert np.array_equal(Z[np.ix_(rows, cols)], ref)
