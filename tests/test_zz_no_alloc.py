"""The allocation-free Beaver matmul entry point against the workspace one.

mpc_beaver_matmul_noalloc exists for callers that cannot allocate device
memory at call time and cannot pass a workspace (their device memory is
reserved by another framework, or they run where allocation calls are not
allowed).  It keeps its scratch in a fixed library-owned device array, so this
test calls it through the C ABI twice in a row, on different inputs, and
checks each result bit for bit against mpc_beaver_matmul (plain engine) on the
same inputs: a stale scratch from the first call must not leak into the
second.  It also checks that an oversized request is refused with MPC_ENOMEM.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("shapes", [[(2, 64, 32, 128), (3, 37, 129, 65)]])
def test_noalloc_matches_workspace_matmul_on_two_calls(mods, shapes):
    mpc, lib = mods
    rng = np.random.default_rng(7)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (P, M, N, K) in enumerate(shapes):
        X, Y = _rand_words(rng, (P, M, K)), _rand_words(rng, (P, K, N))
        A, B, C = mpc.ttp_matmul_triple(P, M, N, K, 1, 500 + call)
        ref = mpc.beaver_matmul(X, Y, A, B, C, algo=mpc.PLAIN, trunc_bits=16)
        Z = torch.full((P, M, N), -1, dtype=torch.int64, device="cuda")
        rc = lib.mpc_beaver_matmul_noalloc(P, M, N, K, _ptr(X), _ptr(Y), _ptr(A), _ptr(B),
                                           _ptr(C), _ptr(Z), 16, stream)
        assert rc == 0, lib.mpc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(Z, ref), f"call {call}: no-alloc result differs"


def test_noalloc_rejects_oversized_request(mods):
    _, lib = mods
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: the size check comes first
    M = N = K = 1024                 # needs 3 Mi words > the 1 Mi-word scratch
    rc = lib.mpc_beaver_matmul_noalloc(2, M, N, K, fake, fake, fake, fake, fake, fake, 16, None)
    assert rc == -3
    assert b"scratch" in lib.mpc_last_error()
