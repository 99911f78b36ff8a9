"""Pins for ring matmul / conv, the dealer and Beaver products (App. D.1.1).

Every expected value here comes from Python's arbitrary-precision integers
reduced mod 2^64 (brute force on tiny shapes) or from the closed-form Beaver
identity reveal(Z) = f(x, y); none re-runs the oracle's own formula.
"""
import numpy as np
import pytest

from oracle import beaver, dealer, fixed, ring, sharing, truncation
from oracle.transcript import Transcript

M64 = (1 << 64) - 1
EDGE = [0, 1, M64, 1 << 63, (1 << 63) - 1, 0x5555555555555555, 0xAAAAAAAAAAAAAAAA, 1 << 32]


def _ints(a):
    return [[int(v) for v in row] for row in np.asarray(a)]


def brute_matmul(a, b):
    A, B = _ints(a), _ints(b)
    M, K, N = len(A), len(B), len(B[0])
    return [[sum(A[i][k] * B[k][j] for k in range(K)) & M64 for j in range(N)] for i in range(M)]


def brute_conv2d(x, w, stride, pad, pad_w=None):
    pad_w = pad if pad_w is None else pad_w
    N, Cin, H, W = x.shape
    Cout, _, kh, kw = w.shape
    Ho = (H + 2 * pad - kh) // stride + 1
    Wo = (W + 2 * pad_w - kw) // stride + 1
    out = np.zeros((N, Cout, Ho, Wo), dtype=object)
    for n in range(N):
        for co in range(Cout):
            for i in range(Ho):
                for j in range(Wo):
                    s = 0
                    for ci in range(Cin):
                        for r in range(kh):
                            for t in range(kw):
                                hi, wi = i * stride + r - pad, j * stride + t - pad_w
                                if 0 <= hi < H and 0 <= wi < W:
                                    s += int(w[co, ci, r, t]) * int(x[n, ci, hi, wi])
                    out[n, co, i, j] = s & M64
    return out


def _u64(rng, shape, edge=True):
    a = rng.integers(0, 2 ** 64, shape, dtype=np.uint64)
    if edge:
        flat = a.reshape(-1)
        flat[: min(len(EDGE), flat.size)] = EDGE[: flat.size]
    return a


@pytest.mark.parametrize("M,K,N", [(1, 1, 1), (3, 5, 2), (8, 8, 8), (7, 1, 9)])
def test_ring_matmul_brute_force(M, K, N, rng):
    a, b = _u64(rng, (M, K)), _u64(rng, (K, N))
    assert _ints(ring.matmul(a, b)) == brute_matmul(a, b)


def test_ring_matmul_all_ones_edge():
    a = np.full((4, 8), M64, dtype=np.uint64)
    b = np.full((8, 3), M64, dtype=np.uint64)
    # (-1)(-1) * 8 = 8
    assert np.all(ring.matmul(a, b) == 8)


@pytest.mark.parametrize("shape,stride,pad", [((1, 2, 5, 5), 1, 1), ((2, 3, 6, 5), 2, 0),
                                              ((1, 1, 4, 7), 2, 1), ((2, 2, 3, 3), 1, 2)])
def test_ring_conv2d_brute_force(shape, stride, pad, rng):
    x = _u64(rng, shape)
    w = _u64(rng, (3, shape[1], 3, 3))
    got = ring.conv2d(x, w, stride, pad)
    assert got.tolist() == brute_conv2d(x, w, stride, pad).tolist()


def test_ring_conv1d_brute_force(rng):
    x = _u64(rng, (1, 3, 17))
    w = _u64(rng, (4, 3, 5))
    got = ring.conv1d(x, w, stride=2, pad=2)
    ref = brute_conv2d(x[:, :, None, :], w[:, :, None, :], 2, 0, pad_w=2)[:, :, 0, :]
    assert got.tolist() == ref.tolist()


@pytest.mark.parametrize("P", [1, 2, 3, 8])
def test_mul_triple_is_a_product(P):
    A, B, C = dealer.mul_triple(P, 50, seed=1, op_id=3)
    a, b, c = (sharing.reveal(t) for t in (A, B, C))
    assert [int(v) for v in c] == [(int(x) * int(y)) & M64 for x, y in zip(a, b)]


def test_matmul_triple_is_a_product():
    A, B, C = dealer.matmul_triple(3, 4, 5, 6, seed=1, op_id=4)
    a, b, c = (sharing.reveal(t) for t in (A, B, C))
    assert _ints(c) == brute_matmul(a, b)


def test_conv_triple_is_a_conv():
    A, B, C = dealer.conv2d_triple(2, (1, 2, 5, 5), (3, 2, 3, 3), 2, 1, seed=1, op_id=5)
    a, b, c = (sharing.reveal(t) for t in (A, B, C))
    assert c.tolist() == brute_conv2d(a, b, 2, 1).tolist()


@pytest.mark.parametrize("P", [1, 2, 3, 4, 8])
def test_beaver_mul_identity(P, rng):
    x, y = _u64(rng, 300), _u64(rng, 300)[::-1].copy()
    X, Y = sharing.share(x, P, 0, 1, 1), sharing.share(y, P, P - 1, 1, 2)
    A, B, C = dealer.mul_triple(P, 300, 1, 3)
    z = sharing.reveal(beaver.beaver_mul(X, Y, A, B, C))
    assert [int(v) for v in z] == [(int(a) * int(b)) & M64 for a, b in zip(x, y)]


@pytest.mark.parametrize("P,M,K,N", [(2, 8, 8, 8), (3, 5, 7, 3), (1, 4, 4, 4), (4, 2, 9, 5)])
def test_beaver_matmul_identity(P, M, K, N, rng):
    x, y = _u64(rng, (M, K)), _u64(rng, (K, N))
    X, Y = sharing.share(x, P, 0, 1, 1), sharing.share(y, P, P - 1, 1, 2)
    A, B, C = dealer.matmul_triple(P, M, N, K, 1, 3)
    assert _ints(sharing.reveal(beaver.beaver_matmul(X, Y, A, B, C))) == brute_matmul(x, y)


def test_beaver_conv2d_identity(rng):
    x, w = _u64(rng, (2, 3, 5, 6)), _u64(rng, (4, 3, 3, 3))
    X, W = sharing.share(x, 2, 0, 1, 1), sharing.share(w, 2, 1, 1, 2)
    A, B, C = dealer.conv2d_triple(2, x.shape, w.shape, 2, 1, 1, 3)
    z = sharing.reveal(beaver.beaver_conv2d(X, W, A, B, C, 2, 1))
    assert z.tolist() == brute_conv2d(x, w, 2, 1).tolist()


def _chi2_bytes(words):
    b = np.asarray(words, dtype=np.uint64).view(np.uint8)
    counts = np.bincount(b, minlength=256)
    e = b.size / 256.0
    return float(((counts - e) ** 2 / e).sum())


def test_opened_values_look_uniform_and_a_bad_dealer_is_caught():
    """App. C / D.1.1: eps = x - a is uniform noise when a is uniform."""
    n = 1 << 14
    x = fixed.encode(np.linspace(-3, 3, n))           # highly structured secret
    X = sharing.share(x, 2, 0, 1, 1)
    A, B, C = dealer.mul_triple(2, n, 1, 3)
    _, eps, _ = beaver.beaver(X, X, A, B, C, lambda u, v: u * v)
    assert _chi2_bytes(eps) < 400
    # Planted mistake (in the oracle, on the CPU): a dealer with a = 0 leaks x.
    _, eps_bad, _ = beaver.beaver(X, X, np.zeros_like(A), B, C, lambda u, v: u * v)
    assert _chi2_bytes(eps_bad) > 1e4


def test_round_count_multiplication_is_one():
    tr = Transcript()
    A, B, C = dealer.mul_triple(2, 8, 1, 1)
    beaver.beaver_mul(A, B, A, B, C, tr)
    assert tr.rounds == 1 and tr.bytes_per_party == 2 * 8 * 8


# --- truncation -----------------------------------------------------------
@pytest.mark.parametrize("divisor", [0, 49, 3])
def test_truncation_two_party_floor(divisor, rng):
    v = rng.integers(-(1 << 43), 1 << 43, 4000)
    S = sharing.share(v.astype(np.int64).view(np.uint64), 2, 0, 7, 7)
    T = truncation.truncate(S, 16, divisor)
    got = sharing.reveal(T).view(np.int64)
    l = divisor or 65536
    fl = np.array([int(a) // l for a in v])      # Python floor division
    d = got - fl
    assert set(np.unique(d).tolist()) <= {-1, 0}


def test_truncation_one_party_is_exact_floor(rng):
    v = rng.integers(-(1 << 62), 1 << 62, 1000).astype(np.int64)
    got = truncation.truncate(v.view(np.uint64)[None], 16)[0].view(np.int64)
    assert got.tolist() == [int(a) >> 16 for a in v]
    got49 = truncation.truncate(v.view(np.uint64)[None], 16, 49)[0].view(np.int64)
    assert got49.tolist() == [int(a) // 49 for a in v]


def test_truncation_costs_no_round():
    tr = Transcript()
    truncation.truncate(np.zeros((2, 4), dtype=np.uint64), 16)
    assert tr.rounds == 0


def test_small_case_fixed_point_error_bound():
    """Closed-form error of dec(trunc(Beaver matmul)) vs the float64 product.

    |err_ij| <= sum_k (|x_ik| + |y_kj|) 2^-17 + K 2^-34 + 2^-15: two encode
    roundings (<= 2^-17 each) and two share floors (error in (-2^-15, 0]).
    The share floors alone average -2^-16: each party's floor drops its share's
    fractional part, and each fractional part is uniform on [0, 1).
    """
    import synth
    X, Y, _, _ = synth.small_case()
    sc = synth.SMALL_SCHEDULE
    x, y = fixed.encode(X), fixed.encode(Y)
    Xs = sharing.share(x, 2, 0, sc["seed"], sc["x_op"])
    Ys = sharing.share(y, 2, 1, sc["seed"], sc["y_op"])
    A, B, C = dealer.matmul_triple(2, 64, 32, 128, sc["seed"], sc["matmul_triple_op"])
    Z = truncation.truncate(beaver.beaver_matmul(Xs, Ys, A, B, C), 16)
    got = fixed.decode(sharing.reveal(Z))
    exact = X @ Y
    bound = (np.abs(X).sum(1)[:, None] + np.abs(Y).sum(0)[None, :]) * 2.0 ** -17 \
        + 128 * 2.0 ** -34 + 2.0 ** -15
    assert np.all(np.abs(got - exact) <= bound)
    # Relative 2^-12 wherever |XY| >= 1.
    big = np.abs(exact) >= 1
    assert np.all(np.abs(got - exact)[big] <= 2.0 ** -12 * np.abs(exact)[big] + bound[big])
    # Truncation part alone: exact ring product v of the encodings.
    v = np.array(brute_matmul(x.view(np.uint64), y.view(np.uint64)), dtype=object)
    vs = np.array([[(int(t) ^ (1 << 63)) - (1 << 63) for t in row] for row in v], dtype=object)
    terr = np.array([[int(g) for g in row] for row in sharing.reveal(Z).view(np.int64)], dtype=object)
    d = np.array([[terr[i, j] * 65536 - vs[i, j] for j in range(32)] for i in range(64)], dtype=float)
    assert d.max() <= 0 and d.min() > -2 * 65536
    assert abs(d.mean() / 65536 + 1.0) < 0.05


# --- n-party truncation (Alg. 1) ---------------------------------------------------
def test_wrap_count_brute_force(rng):
    """theta = (sum_p s(x_p) - s(x)) / Q on tiny hand cases and random shares."""
    Q = 1 << 64
    assert truncation.wrap_count([1, 2]) == 0
    assert truncation.wrap_count([(1 << 63) - 1, 1]) == 1                # 2^63 - 1 + 1 wraps up
    assert truncation.wrap_count([Q - 1, Q - 1]) == 0                    # -1 + -1 = -2
    assert truncation.wrap_count([1 << 63, 1 << 63]) == -1               # -2^63 - 2^63 wraps down
    for _ in range(200):
        sh = [int(v) for v in rng.integers(0, 2 ** 64, 3, dtype=np.uint64)]
        s = [v - Q if v >= 1 << 63 else v for v in sh]
        x = sum(sh) % Q
        xs = x - Q if x >= 1 << 63 else x
        th = truncation.wrap_count(sh)
        assert sum(s) - th * Q == xs and -2 <= th <= 1


def test_trunc_pair_theta_r_is_the_wrap_count():
    R, TH = dealer.trunc_pairs(3, 200, 1, 5)
    th = sharing.reveal(TH).view(np.int64)
    for i in range(200):
        assert th[i] == truncation.wrap_count(R[:, i])


@pytest.mark.parametrize("P", [2, 3, 4, 8])
def test_nparty_truncation_within_p_units(P, rng):
    """Alg. 1 (eta = 0): reveal in [floor(x/l) - (P-1), floor(x/l)] unless x + r wraps."""
    n = 2000
    v = rng.integers(-(1 << 43), 1 << 43, n)
    X = sharing.share(v.astype(np.int64).view(np.uint64), P, 0, 7, 8)
    R, TH = dealer.trunc_pairs(P, n, 7, 9)
    tr = Transcript()
    got = sharing.reveal(truncation.truncate_nparty(X, R, TH, 16, tr)).view(np.int64)
    r = sharing.reveal(R).view(np.int64)
    fl = np.array([int(a) >> 16 for a in v])
    d = got - fl
    # eta != 0 exactly when the signed sum x + r overflows
    eta = np.array([not (-(1 << 63) <= int(a) + int(b) < (1 << 63)) for a, b in zip(v, r)])
    assert np.all((d[~eta] >= -(P - 1)) & (d[~eta] <= 0))
    assert eta.sum() <= 2          # probability about |x| / Q per element
    assert tr.rounds == 1          # Table 3: one round for more than two parties


def test_nparty_truncation_fails_without_wrap_correction(rng):
    """Planted mistake: dropping theta_x (plain local division) breaks P = 3."""
    n = 500
    v = rng.integers(-(1 << 40), 1 << 40, n)
    X = sharing.share(v.astype(np.int64).view(np.uint64), 3, 0, 7, 8)
    naive = sharing.reveal(truncation.truncate(X, 16)).view(np.int64)
    fl = np.array([int(a) >> 16 for a in v])
    assert np.mean(np.abs(naive - fl) > 2) > 0.1   # wraps of three shares are common
