"""A bounded device-side wait that runs out, and the status path behind it.

mpc_test_wait_timeout launches one warp that waits, through the limb engine's
own bounded mbarrier wait and abort flag, for a phase that never completes;
nothing else (no TMA copy, no MMA, no TMEM) is in flight.  After its limit the
kernel records MPC_ETIMEOUT in the device status word and returns.  The test
checks that mpc_sync_status() reports MPC_ETIMEOUT exactly once, then MPC_OK,
and that the next library call (a limb-engine ring GEMM) is still bit-exact
against the oracle: the context stays usable.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OK, ETIMEOUT = 0, -5


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as mpc
    from paper_2109_00984_b300 import _lib
    return mpc, _lib.load()


def test_bounded_wait_runs_out_and_reports_once(mods):
    mpc, lib = mods
    from oracle import ring
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mpc_sync_status(stream) == OK          # start from a clear status word
    assert lib.mpc_test_wait_timeout(1_000_000, stream) == OK     # 1 ms limit
    assert lib.mpc_sync_status(stream) == ETIMEOUT
    assert lib.mpc_sync_status(stream) == OK          # read once, then cleared

    rng = np.random.default_rng(3)
    M, N, K = 200, 136, 300
    Ah = rng.integers(0, 2 ** 64, (M, K), dtype=np.uint64)
    Bh = rng.integers(0, 2 ** 64, (K, N), dtype=np.uint64)
    d = lambda a: torch.from_numpy(a.view(np.int64)).cuda()
    Z = mpc.ring_gemm(d(Ah), d(Bh), None, algo=mpc.LIMB)
    assert lib.mpc_sync_status(stream) == OK
    assert np.array_equal(Z.cpu().numpy().view(np.uint64), ring.matmul(Ah, Bh))


def test_timeout_then_second_timeout_reported_again(mods):
    _, lib = mods
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        assert lib.mpc_test_wait_timeout(50_000, stream) == OK
        assert lib.mpc_sync_status(stream) == ETIMEOUT
    assert lib.mpc_sync_status(stream) == OK
