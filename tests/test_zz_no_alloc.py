"""The allocation-free Beaver matmul entry point against the workspace one.

mpc_beaver_matmul_noalloc exists for callers that cannot allocate device
memory at call time and cannot pass a workspace (their device memory is
reserved by another framework, or they run where allocation calls are not
allowed).  It keeps its scratch in a fixed library-owned device array, so this
test calls it through the C ABI on several shapes in a row, each on fresh
inputs, and checks each result bit for bit against mpc_beaver_matmul (plain
engine) on the same inputs: a stale scratch from an earlier call must not leak
into a later one.  The shapes cover K = 0 (no opening, Z = C truncated),
no truncation, one party, and a request whose rounded scratch is exactly the
array's size; one more is compared with the oracle directly.  The protocol
counters must move by the same amounts for both entry points, and a request 32
words over the array is refused with MPC_ENOMEM.  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCRATCH_WORDS = 1 << 20


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as mpc
    from paper_2109_00984_b300 import _lib
    return mpc, _lib.load()


def _rand_words(rng, shape):
    a = rng.integers(0, 2 ** 64, shape, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).cuda()


def _need(M, N, K):
    r = lambda n: (n + 31) // 32 * 32
    return r(M * K) + 2 * r(K * N)


# (P, M, N, K, trunc_bits), run in this order in one process
SHAPES = [(2, 64, 32, 128, 16), (3, 37, 129, 65, 16), (2, 17, 9, 0, 16), (2, 33, 40, 50, 0),
          (1, 40, 24, 30, 16), (2, 1024, 1536, 256, 16)]
assert _need(1024, 1536, 256) == SCRATCH_WORDS


def test_noalloc_matches_workspace_matmul_on_consecutive_calls(mods):
    mpc, lib = mods
    rng = np.random.default_rng(7)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (P, M, N, K, tb) in enumerate(SHAPES):
        X, Y = _rand_words(rng, (P, M, K)), _rand_words(rng, (P, K, N))
        A, B, C = mpc.ttp_matmul_triple(P, M, N, K, 1, 500 + call)
        mpc.reset_stats()
        ref = mpc.beaver_matmul(X, Y, A, B, C, algo=mpc.PLAIN, trunc_bits=tb)
        torch.cuda.synchronize()
        s_ref = mpc.get_stats()
        Z = torch.full((P, M, N), -1, dtype=torch.int64, device="cuda")
        mpc.reset_stats()
        rc = lib.mpc_beaver_matmul_noalloc(P, M, N, K, _ptr(X), _ptr(Y), _ptr(A), _ptr(B),
                                           _ptr(C), _ptr(Z), tb, stream)
        assert rc == 0, lib.mpc_last_error()
        torch.cuda.synchronize()
        s_new = mpc.get_stats()
        assert torch.equal(Z, ref), f"call {call} {(P, M, N, K, tb)}: no-alloc result differs"
        for key in ("calls", "rounds", "bytes_opened", "triple_words", "ring_macs"):
            assert s_new[key] == s_ref[key], (call, key, s_new[key], s_ref[key])


def test_noalloc_matches_the_oracle(mods):
    mpc, lib = mods
    from oracle import beaver, dealer, truncation
    P, M, N, K = 2, 19, 23, 45
    rng = np.random.default_rng(11)
    Xh = rng.integers(0, 2 ** 64, (P, M, K), dtype=np.uint64)
    Yh = rng.integers(0, 2 ** 64, (P, K, N), dtype=np.uint64)
    oA, oB, oC = dealer.matmul_triple(P, M, N, K, 1, 77)
    ref = truncation.truncate(beaver.beaver_matmul(Xh, Yh, oA, oB, oC), 16)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()
    X, Y, A, B, C = d(Xh), d(Yh), d(oA), d(oB), d(oC)
    Z = torch.empty((P, M, N), dtype=torch.int64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mpc_beaver_matmul_noalloc(P, M, N, K, _ptr(X), _ptr(Y), _ptr(A), _ptr(B), _ptr(C),
                                       _ptr(Z), 16, stream)
    assert rc == 0, lib.mpc_last_error()
    got = Z.cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ref)


def test_noalloc_rejects_oversized_request(mods):
    _, lib = mods
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: the size check comes first
    assert _need(16385, 8192, 32) == SCRATCH_WORDS + 32
    rc = lib.mpc_beaver_matmul_noalloc(2, 16385, 8192, 32, fake, fake, fake, fake, fake, fake, 16,
                                       None)
    assert rc == -3
    assert b"scratch" in lib.mpc_last_error()
    rc = lib.mpc_beaver_matmul_noalloc(2, 1024, 1024, 1024, fake, fake, fake, fake, fake, fake, 16,
                                       None)
    assert rc == -3
