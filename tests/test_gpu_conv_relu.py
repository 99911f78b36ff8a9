"""Beaver convolution + fused private ReLU in one call (mpc_beaver_conv2d_relu).

The composite must equal, word for word, the oracle's Beaver convolution with
truncation followed by its private ReLU on the dealer material at
op .. op + 3, on both engines, for geometries whose GEMM is split along K (the
ReLU kernel then reduces the partial sums, adds C and truncates itself; batch
2 checks the NCHW scatter) and ones that are not split.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, host  # noqa: E402

from oracle import beaver, binary, dealer, truncation  # noqa: E402

SEED = 1

GEOMS = [
    # (batch, c_in, h, w, c_out, k_h, k_w, stride, pad_h, pad_w)
    (1, 64, 1, 200, 24, 1, 7, 1, 0, 3),     # 1-D, split-K on both engines
    (2, 32, 12, 12, 40, 3, 3, 1, 1, 1),     # batch 2 (output scatter), split-K
    (1, 4, 20, 20, 130, 3, 3, 2, 1, 1),     # short K: not split, ragged rows
]


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


@pytest.mark.parametrize("geom", GEOMS)
@pytest.mark.parametrize("engine", ["plain", "limb"])
def test_conv2d_relu_matches_oracle(mpc, geom, engine, rng):
    b, ci, h, w, co, kh, kw, st, ph, pw = geom
    P = 2
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 90, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    n = Z[0].size
    op = 400
    T = dealer.and_triples(P, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(P, n, SEED, op + 1)
    mt = dealer.mul_triple(P, n, SEED, op + 2)
    ref = binary.private_relu(Z.reshape(P, n), T, ra, rb, mt, SEED, op + 3).reshape(Z.shape)

    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    algo = mpc.LIMB if engine == "limb" else mpc.PLAIN
    Y = mpc.beaver_conv2d_relu(dev(X), dev(W), dev(A), dev(B), dev(C), d, SEED, op, algo=algo,
                               trunc_bits=16)
    mpc.sync_status()
    assert np.array_equal(host(Y), ref)
    # the two separate calls give the same words
    Z2 = mpc.beaver_conv2d(dev(X), dev(W), dev(A), dev(B), dev(C), d, algo=algo, trunc_bits=16)
    Y2 = mpc.private_relu_fused(Z2.reshape(P, n), SEED, op).reshape(Y.shape)
    assert torch.equal(Y, Y2)


def test_conv2d_relu_rejects_other_party_counts(mpc):
    from paper_2109_00984_b300 import _lib
    import ctypes
    lib = _lib.load()
    d = mpc.conv_desc(1, 4, 1, 16, 8, 1, 3, 1, 0, 1)
    fake = ctypes.c_void_p(0x1000)
    rc = lib.mpc_beaver_conv2d_relu(3, ctypes.byref(d), fake, fake, fake, fake, fake, fake, 0, 16,
                                    1, 1, fake, 1 << 20, None)
    assert rc == -6


@pytest.mark.parametrize("geom", GEOMS)
def test_prepared_conv2d_relu_matches_oracle(mpc, geom, rng):
    """The convolution split into its input-independent half (prepare: F opened,
    weight-side and im2col(A_p) digit planes) and the online half gives the
    oracle's words, with the ReLU and without it; the prepare call reads no X
    (done before X exists) and the online calls read neither W nor B."""
    b, ci, h, w, co, kh, kw, st, ph, pw = geom
    P = 2
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 91, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    n = Z[0].size
    op = 500
    T = dealer.and_triples(P, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(P, n, SEED, op + 1)
    mt = dealer.mul_triple(P, n, SEED, op + 2)
    ref = binary.private_relu(Z.reshape(P, n), T, ra, rb, mt, SEED, op + 3).reshape(Z.shape)

    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    dA = dev(A)
    prep = mpc.beaver_conv2d_prepare(dev(W), dA, dev(B), d)
    Zp = mpc.beaver_conv2d_prepared(dev(X), dA, dev(C), prep, d, trunc_bits=16)
    Y = mpc.beaver_conv2d_relu_prepared(dev(X), dA, dev(C), prep, d, SEED, op, trunc_bits=16)
    mpc.sync_status()
    assert np.array_equal(host(Zp), Z)
    assert np.array_equal(host(Y), ref)


@pytest.mark.parametrize("P", [3, 8])
def test_prepared_conv2d_more_parties(mpc, P, rng):
    b, ci, h, w, co, kh, kw, st, ph, pw = GEOMS[1]
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 92, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    dA = dev(A)
    prep = mpc.beaver_conv2d_prepare(dev(W), dA, dev(B), d)
    Zp = mpc.beaver_conv2d_prepared(dev(X), dA, dev(C), prep, d, trunc_bits=16)
    mpc.sync_status()
    assert np.array_equal(host(Zp), Z)


@pytest.mark.parametrize("geom", GEOMS)
def test_prepared_products_conv2d_relu_matches_oracle(mpc, geom, rng):
    """The preparation also adds each party's input-independent product A_p F
    into C; the online half is one operand pair per party (E G_p): the oracle's
    words, with the ReLU and without it."""
    b, ci, h, w, co, kh, kw, st, ph, pw = geom
    P = 2
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 93, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    n = Z[0].size
    op = 600
    T = dealer.and_triples(P, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(P, n, SEED, op + 1)
    mt = dealer.mul_triple(P, n, SEED, op + 2)
    ref = binary.private_relu(Z.reshape(P, n), T, ra, rb, mt, SEED, op + 3).reshape(Z.shape)

    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    dA = dev(A)
    prep = mpc.beaver_conv2d_prepare_products(dev(W), dA, dev(B), dev(C), d)
    Zp = mpc.beaver_conv2d_prepared_products(dev(X), dA, prep, d, trunc_bits=16)
    Y = mpc.beaver_conv2d_relu_prepared_products(dev(X), dA, prep, d, SEED, op, trunc_bits=16)
    mpc.sync_status()
    assert np.array_equal(host(Zp), Z)
    assert np.array_equal(host(Y), ref)


@pytest.mark.parametrize("P", [3, 8])
def test_prepared_products_more_parties(mpc, P, rng):
    b, ci, h, w, co, kh, kw, st, ph, pw = GEOMS[1]
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 94, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    dA = dev(A)
    prep = mpc.beaver_conv2d_prepare_products(dev(W), dA, dev(B), dev(C), d)
    Zp = mpc.beaver_conv2d_prepared_products(dev(X), dA, prep, d, trunc_bits=16)
    mpc.sync_status()
    assert np.array_equal(host(Zp), Z)



@pytest.mark.parametrize("geom", GEOMS[:2])
@pytest.mark.parametrize("mode", ["plain", "limb", "prepared"])
def test_conv2d_relu_add_matches_oracle(mpc, geom, mode, rng):
    """Convolution, a residual sum and the ReLU in one call: the oracle's
    truncated Beaver convolution plus S, then its private ReLU."""
    b, ci, h, w, co, kh, kw, st, ph, pw = geom
    P = 2
    xs, wsh = (b, ci, h, w), (co, ci, kh, kw)
    X = rng.integers(0, 2 ** 64, (P,) + xs, dtype=np.uint64)
    W = rng.integers(0, 2 ** 64, (P,) + wsh, dtype=np.uint64)
    A, B, C = dealer.conv2d_triple(P, xs, wsh, st, ph, SEED, 95, pad_w=pw)
    Z = truncation.truncate(beaver.beaver_conv2d(X, W, A, B, C, st, ph, pad_w=pw), 16)
    S = rng.integers(0, 2 ** 64, Z.shape, dtype=np.uint64)
    n = Z[0].size
    op = 650
    T = dealer.and_triples(P, n, 12, SEED, op)
    ra, rb = dealer.b2a_bits(P, n, SEED, op + 1)
    mt = dealer.mul_triple(P, n, SEED, op + 2)
    ref = binary.private_relu((Z + S).reshape(P, n), T, ra, rb, mt, SEED, op + 3).reshape(Z.shape)
    d = mpc.conv_desc(b, ci, h, w, co, kh, kw, st, st, ph, pw)
    if mode == "prepared":
        dA = dev(A)
        prep = mpc.beaver_conv2d_prepare(dev(W), dA, dev(B), d)
        Y = mpc.beaver_conv2d_relu_prepared(dev(X), dA, dev(C), prep, d, SEED, op,
                                            trunc_bits=16, add=dev(S))
    else:
        algo = mpc.LIMB if mode == "limb" else mpc.PLAIN
        Y = mpc.beaver_conv2d_relu(dev(X), dev(W), dev(A), dev(B), dev(C), d, SEED, op,
                                   algo=algo, trunc_bits=16, add=dev(S))
    mpc.sync_status()
    assert np.array_equal(host(Y), ref)
