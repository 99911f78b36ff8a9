"""CPU-only checks of the C ABI: the library loads, exports every declared entry
point, and rejects bad arguments on the host before touching a GPU.

No compute entry point is called with valid arguments here (there is no GPU);
every call below fails validation first, by construction of the ABI.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpc_ring.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2109_00984_b300 import build
    build.build()
    from paper_2109_00984_b300 import _lib
    return _lib.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mpc_ring_share", "mpc_reveal", "mpc_beaver_mul", "mpc_beaver_matmul",
                     "mpc_beaver_conv2d", "mpc_truncate", "mpc_a2b", "mpc_private_relu",
                     "mpc_ttp_mul_triple", "mpc_ttp_matmul_triple", "mpc_ttp_conv2d_triple",
                     "mpc_ttp_and_triples", "mpc_ttp_b2a_bits", "mpc_ring_gemm"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2109_00984_b300 import _lib
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} missing from the Python signature table"


E = dict(OK=0, EINVAL=-1, ERANGE=-2, ENOMEM=-3, ECUDA=-4, ETIMEOUT=-5, EUNSUPPORTED=-6)
NULL = None
FAKE = ctypes.c_void_p(0x1000)   # never dereferenced: every call fails validation first


def test_bad_party_counts_rejected(lib):
    assert lib.mpc_beaver_mul(0, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, NULL, NULL, 0, NULL) == E["EINVAL"]
    assert lib.mpc_beaver_mul(9, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, NULL, NULL, 0, NULL) == E["EINVAL"]
    assert b"party count" in lib.mpc_last_error()
    assert lib.mpc_ring_share(FAKE, 10, 2, 2, 16, 1, 1, FAKE, NULL) == E["EINVAL"]   # src >= P
    assert lib.mpc_private_relu(1, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1, 1, NULL) == E["EUNSUPPORTED"]
    assert lib.mpc_a2b(1, 10, FAKE, FAKE, FAKE, 1, 1, NULL) == E["EUNSUPPORTED"]


def test_null_pointers_rejected(lib):
    assert lib.mpc_beaver_mul(2, 10, FAKE, NULL, FAKE, FAKE, FAKE, FAKE, NULL, NULL, 0, NULL) == E["EINVAL"]
    assert lib.mpc_reveal(FAKE, 2, 10, 16, NULL, NULL, NULL) == E["EINVAL"]
    assert lib.mpc_private_relu(2, 10, FAKE, FAKE, NULL, FAKE, FAKE, FAKE, FAKE, FAKE, 1, 1, NULL) == E["EINVAL"]


def test_bad_sizes_rejected(lib):
    assert lib.mpc_truncate(2, -1, FAKE, 16, 0, NULL) == E["EINVAL"]
    assert lib.mpc_truncate(2, 10, FAKE, 64, 0, NULL) == E["EINVAL"]
    assert lib.mpc_truncate(2, 10, FAKE, 16, -3, NULL) == E["EINVAL"]
    assert lib.mpc_beaver_mul(2, 10, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, NULL, NULL, 64, NULL) == E["EINVAL"]
    assert lib.mpc_beaver_matmul(2, -1, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0, 0, FAKE, 1 << 20, NULL) == E["EINVAL"]
    assert lib.mpc_ring_share(FAKE, 10, 2, 0, 63, 1, 1, FAKE, NULL) == E["EINVAL"]
    assert lib.mpc_ttp_and_triples(2, 10, 0, 1, 1, FAKE, NULL) == E["EINVAL"]
    assert lib.mpc_beaver_matmul(2, 4, 4, 4, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 7, 0, FAKE, 1 << 20, NULL) == E["EINVAL"]


def test_zero_length_is_a_no_op(lib):
    assert lib.mpc_beaver_mul(2, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, 0, NULL) == E["OK"]
    assert lib.mpc_truncate(2, 0, NULL, 16, 0, NULL) == E["OK"]
    assert lib.mpc_private_relu(2, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, 1, 1, NULL) == E["OK"]


def test_workspace_too_small_rejected(lib):
    need = lib.mpc_matmul_workspace_size(2, 64, 32, 128, 0)
    assert need >= 8 * (64 * 128 + 2 * 128 * 32)
    rc = lib.mpc_beaver_matmul(2, 64, 32, 128, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0, 16, FAKE,
                               need - 1, NULL)
    assert rc == E["ENOMEM"]
    assert b"workspace" in lib.mpc_last_error()


def test_conv_descriptor_validation(lib):
    from paper_2109_00984_b300 import _lib
    d = _lib.ConvDesc(1, 3, 5, 5, 4, 7, 7, 1, 1, 0, 0)   # kernel larger than input
    assert lib.mpc_conv2d_workspace_size(2, ctypes.byref(d), 0) == 0
    rc = lib.mpc_beaver_conv2d(2, ctypes.byref(d), FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0, 16, FAKE,
                               1 << 20, NULL)
    assert rc == E["EINVAL"]
    d2 = _lib.ConvDesc(1, 3, 5, 5, 4, 3, 3, 0, 1, 1, 1)  # zero stride
    assert lib.mpc_beaver_conv2d(2, ctypes.byref(d2), FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0, 16,
                                 FAKE, 1 << 20, NULL) == E["EINVAL"]


def test_stats_counters_reset(lib):
    from paper_2109_00984_b300 import _lib
    assert lib.mpc_reset_stats() == 0
    s = _lib.Stats()
    assert lib.mpc_get_stats(ctypes.byref(s)) == 0
    assert s.calls == 0 and s.rounds == 0


def test_shape_products_bounded_before_size_arithmetic(lib):
    from paper_2109_00984_b300 import _lib
    big = 1 << 32   # M*K = K*N = M*N = 2^64 would wrap to 0 if multiplied unchecked
    assert lib.mpc_matmul_workspace_size(2, big, big, big, 0) == 0
    assert lib.mpc_matmul_triple_workspace_size(2, big, big, big, 0) == 0
    assert lib.mpc_ring_gemm_workspace_size(big, big, big, 0) == 0
    assert lib.mpc_beaver_matmul(2, big, big, big, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 0, 0, FAKE,
                                 1 << 40, NULL) == E["EUNSUPPORTED"]
    assert lib.mpc_ring_gemm(big, big, big, FAKE, FAKE, FAKE, FAKE, 0, FAKE, 1 << 40,
                             NULL) == E["EUNSUPPORTED"]
    assert lib.mpc_ttp_matmul_triple(2, big, big, big, 1, 1, FAKE, FAKE, FAKE, 0, FAKE, 1 << 40,
                                     NULL) == E["EUNSUPPORTED"]
    d = _lib.ConvDesc(1 << 20, 1 << 20, 1 << 12, 1 << 12, 4, 1, 1, 1, 1, 0, 0)  # 2^64 data words
    assert lib.mpc_conv2d_workspace_size(2, ctypes.byref(d), 0) == 0
    d = _lib.ConvDesc(1, 3, 5, 5, 1 << 31, 1, 1, 1, 1, 0, 0)                     # field >= 2^31
    assert lib.mpc_conv2d_workspace_size(2, ctypes.byref(d), 0) == 0


def test_noalloc_size_refused_before_any_device_work(lib):
    # The scratch holds 2^20 words.  The refusal must come from the size check,
    # before the device address lookup (which would fail differently here).
    big = 1 << 32
    assert lib.mpc_beaver_matmul_noalloc(2, big, big, big, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 16,
                                         NULL) == E["ENOMEM"]
    assert b"scratch" in lib.mpc_last_error()
    # M*K = 2^19 + 32, 2*K*N = 2^19: 32 words over the scratch.
    assert lib.mpc_beaver_matmul_noalloc(2, 16385, 8192, 32, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                         16, NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_matmul_noalloc(2, 1, 1, (1 << 20) + 1, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                         16, NULL) == E["ENOMEM"]
    # Exactly 2^20 words is accepted by the size check (it then needs a device).
    assert lib.mpc_beaver_matmul_noalloc(2, 16384, 8192, 32, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                         16, NULL) != E["ENOMEM"]


def test_wait_timeout_limit_validated(lib):
    assert lib.mpc_test_wait_timeout(10, NULL) == E["EINVAL"]
    assert lib.mpc_test_wait_timeout(2_000_000_000, NULL) == E["EINVAL"]


def test_prepared_conv_validation(lib):
    from paper_2109_00984_b300 import _lib
    d = _lib.ConvDesc(1, 16, 1, 64, 32, 1, 7, 1, 1, 0, 3)
    need = lib.mpc_conv2d_prep_size(2, ctypes.byref(d))
    K1p = 16 * 7
    assert need >= 16 * K1p * (3 * 32 + 2 * 64)
    assert lib.mpc_conv2d_prep_size(0, ctypes.byref(d)) == 0
    assert lib.mpc_beaver_conv2d_prepare(2, ctypes.byref(d), FAKE, FAKE, FAKE, FAKE, need - 1,
                                         NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_conv2d_prepared(2, ctypes.byref(d), FAKE, FAKE, FAKE, FAKE, need - 1,
                                          FAKE, 16, FAKE, 1 << 20, NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_conv2d_relu_prepared(3, ctypes.byref(d), FAKE, FAKE, FAKE, FAKE, need,
                                               FAKE, 16, 1, 1, FAKE, 1 << 20, NULL) == E["EUNSUPPORTED"]
    assert lib.mpc_beaver_conv2d_prepared(2, ctypes.byref(d), FAKE, FAKE, FAKE, NULL, need,
                                          FAKE, 16, FAKE, 1 << 20, NULL) == E["EINVAL"]


def test_conv_triples_batch_validation(lib):
    from paper_2109_00984_b300 import _lib
    d = _lib.ConvDesc(1, 64, 1, 100, 40, 1, 7, 1, 1, 0, 3)
    # same output shape (40 x 100), other input channels, kernel, stride, padding
    d2 = _lib.ConvDesc(1, 32, 1, 200, 40, 1, 11, 1, 2, 0, 5)
    other = _lib.ConvDesc(1, 64, 1, 100, 48, 1, 7, 1, 1, 0, 3)   # other c_out
    arr = (_lib.ConvDesc * 9)(*([d] * 9))
    one = lib.mpc_conv2d_triple_workspace_size(2, ctypes.byref(d), 1)
    three = lib.mpc_conv2d_triples_workspace_size(2, 3, arr, 1)
    assert 0 < one < three
    assert lib.mpc_conv2d_triples_workspace_size(2, 1, arr, 1) == one
    # the plain engine deals the triples in turn in one triple's workspace
    assert lib.mpc_conv2d_triples_workspace_size(2, 3, arr, 0) == \
        lib.mpc_conv2d_triple_workspace_size(2, ctypes.byref(d), 0)
    for bad in (0, 9):
        assert lib.mpc_conv2d_triples_workspace_size(2, bad, arr, 1) == 0
    mixed = (_lib.ConvDesc * 3)(d, d2, d)
    assert 0 < lib.mpc_conv2d_triples_workspace_size(2, 3, mixed, 1) < three   # d2's K is smaller
    assert lib.mpc_conv2d_triples_workspace_size(2, 3, (_lib.ConvDesc * 3)(d, other, d), 1) == 0
    ids = (ctypes.c_uint64 * 3)(1, 2, 3)
    ptrs = (ctypes.c_void_p * 3)(0x1000, 0x1000, 0x1000)
    holes = (ctypes.c_void_p * 3)(0x1000, None, 0x1000)

    def call(count, descs=arr, op_ids=ids, A=ptrs, ws_bytes=three):
        return lib.mpc_ttp_conv2d_triples(2, count, descs, 1, op_ids, A, ptrs, ptrs, 1, FAKE,
                                          ws_bytes, NULL)
    assert call(0) == E["EINVAL"]
    assert call(9) == E["EINVAL"]
    assert call(3, op_ids=None) == E["EINVAL"]
    assert call(3, A=holes) == E["EINVAL"]
    assert call(3, descs=(_lib.ConvDesc * 3)(d, other, d)) == E["EINVAL"]
    assert call(3, descs=None) == E["EINVAL"]
    assert call(3, ws_bytes=three - 1) == E["ENOMEM"]


def test_prepared_products_validation(lib):
    from paper_2109_00984_b300 import _lib
    d = _lib.ConvDesc(1, 16, 1, 64, 32, 1, 7, 1, 1, 0, 3)
    dp = ctypes.byref(d)
    need = lib.mpc_conv2d_prep_products_size(2, dp)
    K1p = 16 * 7
    assert need >= 2 * (16 * 32 * K1p + 8 * 32 * 64)
    assert lib.mpc_conv2d_prep_products_size(0, dp) == 0
    wneed = lib.mpc_conv2d_prepare_products_workspace_size(2, dp)
    assert wneed > 0
    assert lib.mpc_beaver_conv2d_prepare_products(2, dp, FAKE, FAKE, FAKE, FAKE, FAKE, need - 1,
                                                  FAKE, wneed, NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_conv2d_prepare_products(2, dp, FAKE, FAKE, FAKE, FAKE, FAKE, need,
                                                  FAKE, wneed - 1, NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_conv2d_prepare_products(2, dp, FAKE, FAKE, NULL, FAKE, FAKE, need,
                                                  FAKE, wneed, NULL) == E["EINVAL"]
    assert lib.mpc_beaver_conv2d_prepared_products(2, dp, FAKE, FAKE, FAKE, need - 1, FAKE, 16,
                                                   FAKE, 1 << 30, NULL) == E["ENOMEM"]
    assert lib.mpc_beaver_conv2d_relu_prepared_products(3, dp, FAKE, FAKE, FAKE, need, FAKE, 16,
                                                        1, 1, FAKE, 1 << 30, NULL) == \
        E["EUNSUPPORTED"]

