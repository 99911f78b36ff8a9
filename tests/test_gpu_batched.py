"""Batched Beaver matmul (one persistent launch for many uneven products).

Each product of the batch must equal the oracle's Beaver product with
truncation, word for word, whichever engine the tuning routes it to, also when
the whole call is captured in a CUDA graph and replayed on new inputs.  The
512-product uneven batch (dims log-uniform in [32, 2048], the bench.py
workload) is checked on sampled output blocks, with the oracle regenerating
each sampled product's triple from the PRG streams itself.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, host  # noqa: E402

import synth  # noqa: E402
from oracle import beaver, dealer, prg, ring, sharing, truncation  # noqa: E402

SEED = 1


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def _small_batch(rng, P, count, hi=300):
    dims = rng.integers(1, hi, (count, 3))
    dims[0] = (1, 1, 1)
    dims[1] = (129, 257, 130)
    prods, refs = [], []
    for i, (M, N, K) in enumerate(dims):
        X = rng.integers(0, 2 ** 64, (P, M, K), dtype=np.uint64)
        Y = rng.integers(0, 2 ** 64, (P, K, N), dtype=np.uint64)
        A, B, C = dealer.matmul_triple(P, M, N, K, SEED, 800 + i)
        prods.append((X, Y, A, B, C))
        refs.append(truncation.truncate(beaver.beaver_matmul(X, Y, A, B, C), 16))
    return dims, prods, refs


def _to_dev(prods, P):
    out = []
    for (X, Y, A, B, C) in prods:
        M, N = X.shape[1], Y.shape[2]
        Z = torch.full((P, M, N), -1, dtype=torch.int64, device="cuda")
        out.append((dev(X), dev(Y), dev(A), dev(B), dev(C), Z))
    return out


@pytest.mark.parametrize("P", [1, 2, 3, 8])
@pytest.mark.parametrize("mode", ["plain", "limb", "mixed", "limb_3ctas", "limb_1cta"])
def test_batched_matches_oracle(mpc, P, mode, rng):
    """limb_3ctas / limb_1cta: the persistent limb kernel on 3 CTAs or 1, so
    each CTA runs many tiles of products of different K back to back (the
    barrier phases, chunk counts and TMEM slots carry over between tiles)."""
    dims, prods, refs = _small_batch(rng, P, 17, hi=300 if P < 8 else 140)
    dprods = _to_dev(prods, P)
    tune = mpc.default_tune()
    if mode == "mixed":
        tune.limb_min_macs = float(np.median(dims.prod(1)))   # about half on each engine
    if mode == "limb_3ctas":
        tune.limb_ctas = 3
    if mode == "limb_1cta":
        tune.limb_ctas = 1
    algo = {"plain": mpc.PLAIN, "limb": mpc.LIMB, "mixed": mpc.AUTO, "limb_3ctas": mpc.LIMB,
            "limb_1cta": mpc.LIMB}[mode]
    mpc.beaver_matmul_batched(dprods, algo=algo, trunc_bits=16, tune=tune)
    mpc.sync_status()
    for i, (d, r) in enumerate(zip(dprods, refs)):
        assert np.array_equal(host(d[5]), r), f"product {i} dims {dims[i]}"


def test_batched_graph_replay(mpc, rng):
    """Capture one batched call in a CUDA graph, replay it on fresh inputs."""
    P = 2
    dims, prods, refs = _small_batch(rng, P, 9)
    dprods = _to_dev(prods, P)
    tune = mpc.default_tune()
    tune.limb_min_macs = float(np.median(dims.prod(1)))
    bm = mpc.BatchedMatmul(dprods, algo=mpc.AUTO, trunc_bits=16, tune=tune)
    bm.ensure_workspace()
    bm()                       # warm up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bm()
    torch.cuda.synchronize()
    # New inputs for the same shapes, written into the captured buffers.
    for i, (M, N, K) in enumerate(dims):
        X = rng.integers(0, 2 ** 64, (P, M, K), dtype=np.uint64)
        Y = rng.integers(0, 2 ** 64, (P, K, N), dtype=np.uint64)
        dprods[i][0].copy_(dev(X))
        dprods[i][1].copy_(dev(Y))
        dprods[i][5].fill_(-1)
        A, B, C = prods[i][2:]
        refs[i] = truncation.truncate(beaver.beaver_matmul(X, Y, A, B, C), 16)
    g.replay()
    torch.cuda.synchronize()
    for i, (d, r) in enumerate(zip(dprods, refs)):
        assert np.array_equal(host(d[5]), r), f"replayed product {i}"


def _oracle_block(X, Y, P, M, N, K, op, rows, cols):
    """Oracle Z block for a product whose triple comes from (SEED, op)."""
    oA = np.stack([prg.stream(SEED, op, prg.TRIPLE_A, 0, p, M * K).reshape(M, K) for p in range(P)])
    oB = np.stack([prg.stream(SEED, op, prg.TRIPLE_B, 0, p, K * N).reshape(K, N) for p in range(P)])
    blk = np.ix_(rows, cols)
    with np.errstate(over="ignore"):
        c = ring.matmul(sharing.reveal(oA)[rows], sharing.reveal(oB)[:, cols])
        oC = [prg.stream(SEED, op, prg.TRIPLE_C, 0, p, M * N).reshape(M, N)[blk] for p in range(P - 1)]
        oC.append(c - (sum(oC[1:], oC[0]) if oC else 0))
        E = sharing.reveal(X[:, rows, :] - oA[:, rows, :])
        F = sharing.reveal(Y[:, :, cols] - oB[:, :, cols])
        out = []
        for p in range(P):
            z = oC[p] + ring.matmul(E, oB[p][:, cols]) + ring.matmul(oA[p][rows], F)
            if p == 0:
                z = z + ring.matmul(E, F)
            out.append(truncation.truncate(z, 16))
    return np.stack(out)


@pytest.mark.slow
def test_uneven_512_batch_sampled(mpc):
    """The 512-product uneven batch (seed-2 dims) on the autotuned routing."""
    P = 2
    dims = synth.batched_dims()
    rng = np.random.default_rng(3)
    hostXY, dprods = [], []
    for i, (M, N, K) in enumerate(dims):
        X = rng.integers(0, 2 ** 64, (P, M, K), dtype=np.uint64)
        Y = rng.integers(0, 2 ** 64, (P, K, N), dtype=np.uint64)
        A, B, C = mpc.ttp_matmul_triple(P, int(M), int(N), int(K), SEED, 5000 + i)
        Z = torch.empty((P, M, N), dtype=torch.int64, device="cuda")
        hostXY.append((X, Y))
        dprods.append((dev(X), dev(Y), A, B, C, Z))
    macs = dims.prod(1)
    picks = sorted(set([int(np.argmin(macs)), int(np.argmax(macs))] +
                       [int(i) for i in np.random.default_rng(4).choice(len(dims), 6, replace=False)]))

    def check(label):
        for i in picks:
            M, N, K = (int(v) for v in dims[i])
            r = np.random.default_rng(i)
            rows = np.sort(r.choice(M, min(M, 24), replace=False))
            cols = np.sort(r.choice(N, min(N, 24), replace=False))
            X, Y = hostXY[i]
            ref = _oracle_block(X, Y, P, M, N, K, 5000 + i, rows, cols)
            got = host(dprods[i][5])[:, rows][:, :, cols]
            assert np.array_equal(got, ref), f"{label}: product {i} dims {dims[i]}"

    bm = mpc.BatchedMatmul(dprods, algo=mpc.AUTO, trunc_bits=16)
    bm.autotune()
    bm()
    mpc.sync_status()
    check("autotuned")
    # every product on the persistent limb engine
    for d in dprods:
        d[5].fill_(-1)
    bm = mpc.BatchedMatmul(dprods, algo=mpc.LIMB, trunc_bits=16)
    bm()
    mpc.sync_status()
    check("all limb")


@pytest.mark.parametrize("P", [2, 3])
def test_batched_narrow_edge_tiles(mpc, P, rng):
    """Column counts whose last 128-column tile has at most 64 columns (the
    persistent kernel runs those tiles with N = 64 MMAs) or just over 64, with K
    odd in 16-steps so that the last pass-0 stage holds a single sub-step."""
    dims = np.array([(130, 64, 48), (257, 65, 80), (96, 192, 112), (140, 200, 16),
                     (64, 129, 272), (200, 320, 208), (33, 1, 144)])
    prods, refs = [], []
    for i, (M, N, K) in enumerate(dims):
        X = rng.integers(0, 2 ** 64, (P, M, K), dtype=np.uint64)
        Y = rng.integers(0, 2 ** 64, (P, K, N), dtype=np.uint64)
        A, B, C = dealer.matmul_triple(P, M, N, K, SEED, 900 + i)
        prods.append((X, Y, A, B, C))
        refs.append(truncation.truncate(beaver.beaver_matmul(X, Y, A, B, C), 16))
    dprods = _to_dev(prods, P)
    tune = mpc.default_tune()
    tune.limb_ctas = 5
    mpc.beaver_matmul_batched(dprods, algo=mpc.LIMB, trunc_bits=16, tune=tune)
    mpc.sync_status()
    for i, (d, r) in enumerate(zip(dprods, refs)):
        assert np.array_equal(host(d[5]), r), f"product {i} dims {dims[i]}"
