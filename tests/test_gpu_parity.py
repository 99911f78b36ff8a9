"""GPU parity: every entry point of the C ABI against the CPU oracle, bit-exact.

Everything on this path is integer arithmetic modulo 2^64 (the single float
step, encoding, is one correctly-rounded rint in both implementations), so the
bar is equality of every share word.  Sizes span several tiles and a ragged
tail; the degenerate cases (n = 0, one party, 2^63, all-ones) are included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, dev_f64, host, unpack_bits  # noqa: E402

from oracle import beaver, binary, dealer, fixed, ring, sharing, truncation  # noqa: E402

M64 = (1 << 64) - 1
SEED = 1


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def u64(rng, shape):
    a = rng.integers(0, 2 ** 64, shape, dtype=np.uint64)
    flat = a.reshape(-1)
    edge = [0, 1, M64, 1 << 63, (1 << 63) - 1, 0xFF00FF00FF00FF00]
    flat[: min(len(edge), flat.size)] = edge[: flat.size]
    return a


# ---- sharing / reveal -----------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 3, 8])
@pytest.mark.parametrize("n", [1, 5, 4096, 100003])
def test_ring_share_bit_exact(mpc, P, n, rng):
    x = rng.uniform(-1000, 1000, n)
    src = P - 1
    got = host(mpc.ring_share(dev_f64(x), P, src, SEED, 77))
    ref = sharing.share(fixed.encode(x), P, src, SEED, 77)
    assert np.array_equal(got, ref)


def test_ring_share_encoded_bit_exact(mpc, rng):
    x = u64(rng, 1001)
    got = host(mpc.ring_share_encoded(dev(x), 3, 1, SEED, 5))
    assert np.array_equal(got, sharing.share(x, 3, 1, SEED, 5))


def test_ring_share_range_error(mpc):
    x = dev_f64(np.array([1.0, 2.0 ** 47, 3.0]))
    mpc.ring_share(x, 2, 0, SEED, 1)
    with pytest.raises(mpc.MPCError) as ei:
        mpc.sync_status()
    assert ei.value.code == -2
    mpc.sync_status()   # cleared


@pytest.mark.parametrize("P", [1, 2, 5])
def test_reveal(mpc, P, rng):
    S = u64(rng, (P, 3001))
    r, f = mpc.reveal(dev(S), 16, ring=True, real=True)
    v = sharing.reveal(S)
    assert np.array_equal(host(r), v)
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), fixed.decode(v))


# ---- dealer ------------------------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 3, 8])
def test_mul_triple(mpc, P):
    n = 4099
    A, B, C = mpc.ttp_mul_triple(P, n, SEED, 11)
    rA, rB, rC = dealer.mul_triple(P, n, SEED, 11)
    assert np.array_equal(host(A), rA) and np.array_equal(host(B), rB)
    assert np.array_equal(host(C), rC)


@pytest.mark.parametrize("P", [2, 3])
def test_and_triples(mpc, P):
    n = 1027
    T = mpc.ttp_and_triples(P, n, SEED, 12)
    assert np.array_equal(host(T), dealer.and_triples(P, n, 12, SEED, 12))


@pytest.mark.parametrize("P,n", [(2, 1), (2, 200), (3, 4096), (2, 64 * 37 + 5)])
def test_b2a_bits(mpc, P, n):
    ra, rb = mpc.ttp_b2a_bits(P, n, SEED, 13)
    ora, orb = dealer.b2a_bits(P, n, SEED, 13)
    assert np.array_equal(host(ra), ora)
    words = host(rb)
    assert np.array_equal(unpack_bits(words, n), orb)
    # unused tail bits are zero
    tail = n % 64
    if tail:
        assert not np.any(words[:, -1] >> np.uint64(tail))


@pytest.mark.parametrize("P,M,N,K", [(2, 64, 32, 128), (3, 65, 33, 130), (1, 1, 1, 1),
                                     (2, 129, 257, 7)])
def test_matmul_triple(mpc, P, M, N, K):
    A, B, C = mpc.ttp_matmul_triple(P, M, N, K, SEED, 14)
    rA, rB, rC = dealer.matmul_triple(P, M, N, K, SEED, 14)
    assert np.array_equal(host(A), rA) and np.array_equal(host(B), rB)
    assert np.array_equal(host(C), rC)


def test_conv_triple(mpc):
    d = mpc.conv_desc(2, 3, 9, 7, 5, 3, 3, 2, 2, 1, 1)
    A, B, C = mpc.ttp_conv2d_triple(2, d, SEED, 15)
    rA, rB, rC = dealer.conv2d_triple(2, (2, 3, 9, 7), (5, 3, 3, 3), 2, 1, SEED, 15)
    assert np.array_equal(host(A), rA) and np.array_equal(host(B), rB)
    assert np.array_equal(host(C), rC)


# ---- online -------------------------------------------------------------------------
@pytest.mark.parametrize("P", [1, 2, 3, 8])
@pytest.mark.parametrize("trunc", [0, 16])
def test_beaver_mul(mpc, P, trunc, rng):
    n = 10007
    X, Y = u64(rng, (P, n)), u64(rng, (P, n))
    A, B, C = dealer.mul_triple(P, n, SEED, 21)
    E = torch.empty(n, dtype=torch.int64, device="cuda")
    F = torch.empty(n, dtype=torch.int64, device="cuda")
    Z = mpc.beaver_mul(dev(X), dev(Y), dev(A), dev(B), dev(C), trunc_bits=trunc, E_out=E, F_out=F)
    ref, eps, delta = beaver.beaver(X, Y, A, B, C, lambda u, v: u * v)
    if trunc:
        ref = truncation.truncate(ref, trunc)
    assert np.array_equal(host(Z), ref)
    assert np.array_equal(host(E), eps) and np.array_equal(host(F), delta)


def test_beaver_mul_small_case_elementwise(mpc):
    import synth
    _, _, xe, ye = synth.small_case()
    sc = synth.SMALL_SCHEDULE
    X = mpc.ring_share(dev_f64(xe), 2, 0, sc["seed"], sc["xe_op"])
    Y = mpc.ring_share(dev_f64(ye), 2, 1, sc["seed"], sc["ye_op"])
    A, B, C = mpc.ttp_mul_triple(2, 4096, sc["seed"], sc["mul_triple_op"])
    Z = mpc.beaver_mul(X, Y, A, B, C, trunc_bits=16)
    oX = sharing.share(fixed.encode(xe), 2, 0, sc["seed"], sc["xe_op"])
    oY = sharing.share(fixed.encode(ye), 2, 1, sc["seed"], sc["ye_op"])
    oA, oB, oC = dealer.mul_triple(2, 4096, sc["seed"], sc["mul_triple_op"])
    ref = truncation.truncate(beaver.beaver_mul(oX, oY, oA, oB, oC), 16)
    assert np.array_equal(host(Z), ref)


@pytest.mark.parametrize("divisor", [0, 49])
def test_truncate(mpc, divisor, rng):
    S = u64(rng, (2, 5003))
    got = host(mpc.truncate(dev(S), 16, divisor))
    assert np.array_equal(got, truncation.truncate(S, 16, divisor))


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (7, 9, 3), (128, 128, 8), (129, 257, 130),
                                   (300, 70, 513)])
def test_ring_gemm_plain(mpc, M, N, K, rng):
    a, b, c = u64(rng, (M, K)), u64(rng, (K, N)), u64(rng, (M, N))
    Z = mpc.ring_gemm(dev(a), dev(b), dev(c), algo=mpc.PLAIN)
    with np.errstate(over="ignore"):
        assert np.array_equal(host(Z), ring.matmul(a, b) + c)
    Z0 = mpc.ring_gemm(dev(a), dev(b), None, algo=mpc.PLAIN)
    assert np.array_equal(host(Z0), ring.matmul(a, b))


def test_small_case_matmul(mpc):
    """The 64x128 . 128x32 two-party product with truncation, end to end."""
    import synth
    Xr, Yr, _, _ = synth.small_case()
    sc = synth.SMALL_SCHEDULE
    X = mpc.ring_share(dev_f64(Xr), 2, 0, sc["seed"], sc["x_op"])
    Y = mpc.ring_share(dev_f64(Yr), 2, 1, sc["seed"], sc["y_op"])
    A, B, C = mpc.ttp_matmul_triple(2, 64, 32, 128, sc["seed"], sc["matmul_triple_op"])
    Z = mpc.beaver_matmul(X, Y, A, B, C, algo=mpc.PLAIN, trunc_bits=16)
    oX = sharing.share(fixed.encode(Xr), 2, 0, sc["seed"], sc["x_op"])
    oY = sharing.share(fixed.encode(Yr), 2, 1, sc["seed"], sc["y_op"])
    oA, oB, oC = dealer.matmul_triple(2, 64, 32, 128, sc["seed"], sc["matmul_triple_op"])
    ref = truncation.truncate(beaver.beaver_matmul(oX, oY, oA, oB, oC), 16)
    assert np.array_equal(host(Z), ref)
    _, real = mpc.reveal(Z)
    torch.cuda.synchronize()
    assert np.max(np.abs(real.cpu().numpy() - Xr @ Yr)) < 2.0 ** -7


@pytest.mark.parametrize("P,M,N,K,trunc", [(3, 65, 33, 130, 0), (2, 129, 200, 257, 16),
                                           (4, 5, 3, 2, 16), (1, 40, 40, 40, 0)])
def test_beaver_matmul_plain(mpc, P, M, N, K, trunc, rng):
    X, Y = u64(rng, (P, M, K)), u64(rng, (P, K, N))
    A, B, C = dealer.matmul_triple(P, M, N, K, SEED, 31)
    Z = mpc.beaver_matmul(dev(X), dev(Y), dev(A), dev(B), dev(C), algo=mpc.PLAIN, trunc_bits=trunc)
    ref = beaver.beaver_matmul(X, Y, A, B, C)
    if trunc:
        ref = truncation.truncate(ref, trunc)
    assert np.array_equal(host(Z), ref)


@pytest.mark.parametrize("geom", [
    dict(batch=2, c_in=3, h=9, w=7, c_out=5, k=3, stride=2, pad=1),
    dict(batch=1, c_in=4, h=8, w=8, c_out=130, k=1, stride=1, pad=0),
    dict(batch=3, c_in=2, h=5, w=6, c_out=4, k=5, stride=1, pad=2),
])
@pytest.mark.parametrize("P", [2, 3])
def test_beaver_conv2d_plain(mpc, geom, P, rng):
    g = geom
    d = mpc.conv_desc(g["batch"], g["c_in"], g["h"], g["w"], g["c_out"], g["k"], g["k"],
                      g["stride"], g["stride"], g["pad"], g["pad"])
    xs = (g["batch"], g["c_in"], g["h"], g["w"])
    ws = (g["c_out"], g["c_in"], g["k"], g["k"])
    X, W = u64(rng, (P,) + xs), u64(rng, (P,) + ws)
    A, B, C = dealer.conv2d_triple(P, xs, ws, g["stride"], g["pad"], SEED, 32)
    Z = mpc.beaver_conv2d(dev(X), dev(W), dev(A), dev(B), dev(C), d, algo=mpc.PLAIN, trunc_bits=16)
    ref = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, g["stride"], g["pad"]), 16)
    assert np.array_equal(host(Z), ref)


def test_beaver_conv1d_speech_geometry(mpc, rng):
    """First speech layer geometry, shortened: k = 11, stride 2, pad 5."""
    L, Cin, Cout = 203, 5, 24
    d = mpc.conv_desc(1, Cin, 1, L, Cout, 1, 11, 1, 2, 0, 5)
    X, W = u64(rng, (2, 1, Cin, 1, L)), u64(rng, (2, Cout, Cin, 1, 11))
    A, B, C = dealer.conv2d_triple(2, (1, Cin, 1, L), (Cout, Cin, 1, 11), 2, 0, SEED, 33, pad_w=5)
    Z = mpc.beaver_conv2d(dev(X), dev(W), dev(A), dev(B), dev(C), d, algo=mpc.PLAIN, trunc_bits=16)
    ref = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, 2, 0, pad_w=5), 16)
    assert np.array_equal(host(Z), ref)


# ---- binary --------------------------------------------------------------------------
@pytest.mark.parametrize("n", [1, 3, 4096, 50001])
def test_a2b(mpc, n, rng):
    X = u64(rng, (2, n))
    T = dealer.and_triples(2, n, 12, SEED, 41)
    got = host(mpc.a2b(dev(X), dev(T), SEED, 42))
    ref = binary.a2b(X, T, SEED, 42)
    assert np.array_equal(got, ref)
    x = sharing.reveal(X)
    assert np.array_equal(sharing.reveal_xor(got), x)


@pytest.mark.parametrize("n", [1, 7, 4096, 65 * 64 + 3, 200001])
def test_private_relu(mpc, n, rng):
    v = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    v[: min(4, n)] = [0, 1, -1, 65536][: min(4, n)]
    X = sharing.share(v.view(np.uint64), 2, 0, SEED, 51)
    T = dealer.and_triples(2, n, 12, SEED, 52)
    ra, rb = dealer.b2a_bits(2, n, SEED, 53)
    mt = dealer.mul_triple(2, n, SEED, 54)
    gra, grb = mpc.ttp_b2a_bits(2, n, SEED, 53)
    got = host(mpc.private_relu(dev(X), dev(T), gra, grb, tuple(dev(t) for t in mt), SEED, 55))
    ref = binary.private_relu(X, T, ra, rb, mt, SEED, 55)
    assert np.array_equal(got, ref)
    assert sharing.reveal(got).view(np.int64).tolist() == np.maximum(v, 0).tolist()


def test_stats_round_counts(mpc):
    """Table 3: multiplication 1 round, A2B 7 (two parties), B2A 1, truncation 0."""
    n = 64
    mpc.reset_stats()
    A, B, C = mpc.ttp_mul_triple(2, n, SEED, 1)
    mpc.beaver_mul(A, B, A, B, C)
    assert mpc.get_stats()["rounds"] == 1
    mpc.truncate(A)
    assert mpc.get_stats()["rounds"] == 1
    T = mpc.ttp_and_triples(2, n, SEED, 2)
    mpc.a2b(A, T, SEED, 3)
    assert mpc.get_stats()["rounds"] == 8
    ra, rb = mpc.ttp_b2a_bits(2, n, SEED, 4)
    MT = torch.stack([A, B, C])
    mpc.private_relu(A, T, ra, rb, MT, SEED, 5)
    s = mpc.get_stats()
    assert s["rounds"] == 8 + 9
    assert s["and_gates"] == 2 * 12 * n


# ---- n-party truncation (Alg. 1) -------------------------------------------------------
@pytest.mark.parametrize("P", [2, 3, 4])
def test_trunc_pairs(mpc, P):
    n = 1003
    r, th = mpc.ttp_trunc_pairs(P, n, SEED, 90)
    oR, oTH = dealer.trunc_pairs(P, n, SEED, 90)
    assert np.array_equal(host(r), oR) and np.array_equal(host(th), oTH)


@pytest.mark.parametrize("P", [2, 3, 4, 8])
def test_truncate_nparty(mpc, P, rng):
    n = 3001
    v = rng.integers(-(1 << 43), 1 << 43, n)
    v[:3] = [0, -1, (1 << 43) - 1]
    X = sharing.share(v.astype(np.int64).view(np.uint64), P, 0, SEED, 91)
    oR, oTH = dealer.trunc_pairs(P, n, SEED, 92)
    got = host(mpc.truncate_nparty(dev(X), dev(oR), dev(oTH), 16))
    assert np.array_equal(got, truncation.truncate_nparty(X, oR, oTH, 16))


def test_three_party_fixed_point_matmul(mpc):
    """P = 3: Beaver matmul, then Alg. 1 truncation; decoded error within the bound."""
    import synth
    Xr, Yr, _, _ = synth.small_case()
    P, seed = 3, 1
    X = mpc.ring_share(dev_f64(Xr), P, 0, seed, 201)
    Y = mpc.ring_share(dev_f64(Yr), P, 2, seed, 202)
    A, B, C = mpc.ttp_matmul_triple(P, 64, 32, 128, seed, 203)
    Z = mpc.beaver_matmul(X, Y, A, B, C, algo=mpc.PLAIN, trunc_bits=0)
    r, th = mpc.ttp_trunc_pairs(P, 64 * 32, seed, 204)
    mpc.truncate_nparty(Z, r, th, 16)
    oX = sharing.share(fixed.encode(Xr), P, 0, seed, 201)
    oY = sharing.share(fixed.encode(Yr), P, 2, seed, 202)
    oA, oB, oC = dealer.matmul_triple(P, 64, 32, 128, seed, 203)
    oZ = beaver.beaver_matmul(oX, oY, oA, oB, oC).reshape(P, -1)
    oR, oTH = dealer.trunc_pairs(P, 64 * 32, seed, 204)
    ref = truncation.truncate_nparty(oZ, oR, oTH, 16)
    got = host(Z).reshape(P, -1)
    assert np.array_equal(got, ref)
    real = fixed.decode(sharing.reveal(got)).reshape(64, 32)
    bound = (np.abs(Xr).sum(1)[:, None] + np.abs(Yr).sum(0)[None, :]) * 2.0 ** -17 \
        + 128 * 2.0 ** -34 + P * 2.0 ** -16
    assert np.all(np.abs(real - Xr @ Yr) <= bound)


# ---- A2B / ReLU for more than two parties (adder tree) ---------------------------------
@pytest.mark.parametrize("P", [3, 4, 5, 8])
def test_a2b_adder_tree(mpc, P, rng):
    n = 1031
    X = u64(rng, (P, n))
    T = dealer.and_triples(P, n, 12 * (P - 1), SEED, 93)
    got = host(mpc.a2b(dev(X), dev(T), SEED, 94))
    assert np.array_equal(got, binary.a2b(X, T, SEED, 94))


@pytest.mark.parametrize("P", [3, 4])
def test_private_relu_adder_tree(mpc, P, rng):
    n = 777
    v = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    v[:3] = [0, 1, -1]
    X = sharing.share(v.view(np.uint64), P, 0, SEED, 95)
    T = dealer.and_triples(P, n, 12 * (P - 1), SEED, 96)
    ra, rb = dealer.b2a_bits(P, n, SEED, 97)
    mt = dealer.mul_triple(P, n, SEED, 98)
    gra, grb = mpc.ttp_b2a_bits(P, n, SEED, 97)
    got = host(mpc.private_relu(dev(X), dev(T), gra, grb, tuple(dev(t) for t in mt), SEED, 99))
    assert np.array_equal(got, binary.private_relu(X, T, ra, rb, mt, SEED, 99))
    assert sharing.reveal(got).view(np.int64).tolist() == np.maximum(v, 0).tolist()


@pytest.mark.parametrize("n", [1, 7, 4096, 65 * 64 + 3, 200001])
def test_private_relu_fused_dealer(mpc, n, rng):
    """Dealer regenerated in registers: identical to the separate dealer calls."""
    v = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    v[: min(3, n)] = [0, 1, -1][: min(3, n)]
    X = sharing.share(v.view(np.uint64), 2, 0, SEED, 61)
    op = 700
    T = dealer.and_triples(2, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(2, n, SEED, op + 1)
    mt = dealer.mul_triple(2, n, SEED, op + 2)
    ref = binary.private_relu(X, T, ra, rb, mt, SEED, op + 3)
    got = host(mpc.private_relu_fused(dev(X), SEED, op))
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n", [1, 1000, 50001])
def test_private_relu_fused_add(mpc, n, rng):
    """ReLU of a sum of two sharings (a residual connection) in one kernel: the
    oracle's private addition then its private ReLU, word for word."""
    v = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    u = rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64)
    X = sharing.share(v.view(np.uint64), 2, 0, SEED, 62)
    S = sharing.share(u.view(np.uint64), 2, 1, SEED, 63)
    op = 720
    T = dealer.and_triples(2, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(2, n, SEED, op + 1)
    mt = dealer.mul_triple(2, n, SEED, op + 2)
    ref = binary.private_relu(X + S, T, ra, rb, mt, SEED, op + 3)
    got = host(mpc.private_relu_fused(dev(X), SEED, op, add=dev(S)))
    assert np.array_equal(got, ref)
    # in place over X
    dX = dev(X)
    mpc.private_relu_fused(dX, SEED, op, out=dX, add=dev(S))
    assert np.array_equal(host(dX), ref)


def test_private_max_fused_slices(mpc, rng):
    """max(A_i, B_i) = B_i + ReLU(A_i - B_i) pair by pair, each slice taking the
    material of its elements in one batched ReLU over both pairs: the oracle's
    subtraction, one private ReLU over the batch, and addition, word for word."""
    n = 1000
    A = [sharing.share(rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64).view(np.uint64),
                       2, 0, SEED, 70 + i) for i in range(2)]
    B = [sharing.share(rng.integers(-(1 << 40), 1 << 40, n).astype(np.int64).view(np.uint64),
                       2, 1, SEED, 80 + i) for i in range(2)]
    op = 740
    D = np.concatenate([A[i] - B[i] for i in range(2)], axis=1)
    T = dealer.and_triples(2, 2 * n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(2, 2 * n, SEED, op + 1)
    mt = dealer.mul_triple(2, 2 * n, SEED, op + 2)
    R = binary.private_relu(D, T, ra, rb, mt, SEED, op + 3)
    for i in range(2):
        got = host(mpc.private_max_fused(dev(A[i]), dev(B[i]), SEED, op, elem_offset=i * n))
        assert np.array_equal(got, B[i] + R[:, i * n:(i + 1) * n])
    with pytest.raises(mpc.MPCError):
        mpc.private_max_fused(dev(A[0]), dev(B[0]), SEED, op, elem_offset=3)


# ---- square, affine, comparators, multiplexing ----------------------------------------
@pytest.mark.parametrize("P", [1, 2, 3])
def test_beaver_square(mpc, P, rng):
    n = 5001
    X = u64(rng, (P, n))
    A, B = mpc.ttp_square_pair(P, n, SEED, 301)
    oA, oB = dealer.square_pair(P, n, SEED, 301)
    assert np.array_equal(host(A), oA) and np.array_equal(host(B), oB)
    got = host(mpc.beaver_square(dev(X), A, B, trunc_bits=16))
    assert np.array_equal(got, truncation.truncate(beaver.beaver_square(X, oA, oB), 16))


def test_affine(mpc, rng):
    X = u64(rng, (3, 777))
    got = host(mpc.affine(dev(X), -7, 99, trunc_bits=3))
    assert np.array_equal(got, beaver.affine(X, -7, 99, trunc_bits=3))


@pytest.mark.parametrize("P", [2, 3])
def test_comparators(mpc, P, rng):
    from oracle import compare
    a = rng.integers(-50, 50, 600) * 65536
    b = rng.integers(-50, 50, 600) * 65536
    b[:150] = a[:150]
    X = sharing.share(a.astype(np.int64).view(np.uint64), P, 0, SEED, 5)
    Y = sharing.share(b.astype(np.int64).view(np.uint64), P, P - 1, SEED, 6)
    for name in ("lt", "gt", "ge", "le", "eq", "ne"):
        got = host(getattr(mpc, name)(dev(X), dev(Y), SEED, 3000))
        assert np.array_equal(got, getattr(compare, name)(X, Y, SEED, 3000)), name


def test_mux(mpc, rng):
    from oracle import compare
    c = rng.integers(0, 2, 900).astype(np.int64)
    Cs = sharing.share(c.view(np.uint64), 2, 0, SEED, 9)
    X, Y = u64(rng, (2, 900)), u64(rng, (2, 900))
    got = host(mpc.mux(dev(Cs), dev(X), dev(Y), SEED, 4000))
    assert np.array_equal(got, compare.mux(Cs, X, Y, SEED, 4000))
