"""ctypes loader for libmpcring.so: signatures of every entry point in mpc_ring.h.

The library is built in-tree (``python -m paper_2109_00984_b300.build``); there is
no fallback: if the shared object is missing or fails to load, importing the
package raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpcring.so")

c_int, c_i64, c_u64, c_size, c_vp, c_dp = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                           ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class ConvDesc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "batch", "c_in", "h", "w", "c_out", "kh", "kw", "stride_h", "stride_w", "pad_h", "pad_w")]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "calls", "rounds", "bytes_opened", "and_gates", "triple_words", "ring_macs", "launches")]


class MatmulDesc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int64), ("N", ctypes.c_int64), ("K", ctypes.c_int64)] + \
        [(n, ctypes.c_void_p) for n in ("X", "Y", "A", "B", "C", "Z")]


class Tune(ctypes.Structure):
    _fields_ = [("limb_min_macs", ctypes.c_double), ("persistent_ctas", ctypes.c_int),
                ("limb_ctas", ctypes.c_int)]


_P = ctypes.POINTER
SIGNATURES = {
    "mpc_last_error": (ctypes.c_char_p, []),
    "mpc_sync_status": (c_int, [c_vp]),
    "mpc_get_stats": (c_int, [_P(Stats)]),
    "mpc_reset_stats": (c_int, []),
    "mpc_profile_enable": (c_int, [c_int]),
    "mpc_profile_reset": (c_int, []),
    "mpc_profile_read": (c_int, [ctypes.c_char_p, _P(ctypes.c_uint64), _P(ctypes.c_double)]),
    "mpc_profile_busy": (c_int, [ctypes.c_char_p, _P(ctypes.c_double)]),
    "mpc_test_wait_timeout": (c_int, [c_i64, c_vp]),
    "mpc_ring_share": (c_int, [c_vp, c_i64, c_int, c_int, c_int, c_u64, c_u64, c_vp, c_vp]),
    "mpc_ring_share_encoded": (c_int, [c_vp, c_i64, c_int, c_int, c_u64, c_u64, c_vp, c_vp]),
    "mpc_reveal": (c_int, [c_vp, c_int, c_i64, c_int, c_vp, c_vp, c_vp]),
    "mpc_ttp_mul_triple": (c_int, [c_int, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp, c_vp]),
    "mpc_matmul_triple_workspace_size": (c_size, [c_int, c_i64, c_i64, c_i64, c_int]),
    "mpc_ttp_matmul_triple": (c_int, [c_int, c_i64, c_i64, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp,
                                      c_int, c_vp, c_size, c_vp]),
    "mpc_conv2d_triple_workspace_size": (c_size, [c_int, _P(ConvDesc), c_int]),
    "mpc_ttp_conv2d_triple": (c_int, [c_int, _P(ConvDesc), c_u64, c_u64, c_vp, c_vp, c_vp, c_int,
                                      c_vp, c_size, c_vp]),
    "mpc_conv2d_triples_workspace_size": (c_size, [c_int, c_int, _P(ConvDesc), c_int]),
    "mpc_ttp_conv2d_triples": (c_int, [c_int, c_int, _P(ConvDesc), c_u64, _P(c_u64), _P(c_vp),
                                       _P(c_vp), _P(c_vp), c_int, c_vp, c_size, c_vp]),
    "mpc_ttp_and_triples": (c_int, [c_int, c_i64, c_int, c_u64, c_u64, c_vp, c_vp]),
    "mpc_ttp_b2a_bits": (c_int, [c_int, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp]),
    "mpc_beaver_mul": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_int,
                               c_vp]),
    "mpc_matmul_workspace_size": (c_size, [c_int, c_i64, c_i64, c_i64, c_int]),
    "mpc_beaver_matmul": (c_int, [c_int, c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                  c_int, c_int, c_vp, c_size, c_vp]),
    "mpc_beaver_matmul_noalloc": (c_int, [c_int, c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp,
                                          c_vp, c_int, c_vp]),
    "mpc_conv2d_workspace_size": (c_size, [c_int, _P(ConvDesc), c_int]),
    "mpc_beaver_conv2d_relu": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                       c_int, c_int, c_u64, c_u64, c_vp, c_size, c_vp]),
    "mpc_beaver_conv2d": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_int,
                                  c_int, c_vp, c_size, c_vp]),
    "mpc_conv2d_prep_size": (c_size, [c_int, _P(ConvDesc)]),
    "mpc_beaver_conv2d_prepare": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp, c_size,
                                          c_vp]),
    "mpc_beaver_conv2d_prepared": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp, c_size,
                                           c_vp, c_int, c_vp, c_size, c_vp]),
    "mpc_beaver_conv2d_relu_prepared": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp,
                                                c_size, c_vp, c_int, c_u64, c_u64, c_vp, c_size,
                                                c_vp]),
    "mpc_conv2d_prep_products_size": (c_size, [c_int, _P(ConvDesc)]),
    "mpc_conv2d_prepare_products_workspace_size": (c_size, [c_int, _P(ConvDesc)]),
    "mpc_beaver_conv2d_prepare_products": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp,
                                                   c_vp, c_size, c_vp, c_size, c_vp]),
    "mpc_beaver_conv2d_prepared_products": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_size,
                                                    c_vp, c_int, c_vp, c_size, c_vp]),
    "mpc_beaver_conv2d_relu_prepared_products": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp,
                                                         c_size, c_vp, c_int, c_u64, c_u64, c_vp,
                                                         c_size, c_vp]),
    "mpc_beaver_conv2d_relu_add": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp, c_vp,
                                           c_vp, c_vp, c_int, c_int, c_u64, c_u64, c_vp, c_size,
                                           c_vp]),
    "mpc_beaver_conv2d_relu_prepared_add": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp, c_vp,
                                                    c_size, c_vp, c_vp, c_int, c_u64, c_u64,
                                                    c_vp, c_size, c_vp]),
    "mpc_tune_default": (c_int, [_P(Tune)]),
    "mpc_matmul_batched_workspace_size": (c_size, [c_int, c_int, _P(MatmulDesc), c_int, _P(Tune)]),
    "mpc_beaver_matmul_batched": (c_int, [c_int, c_int, _P(MatmulDesc), c_int, _P(Tune), c_int,
                                          c_vp, c_size, c_vp]),
    "mpc_autotune_batched": (c_int, [c_int, c_int, _P(MatmulDesc), c_int, c_vp, c_size, c_vp,
                                     _P(Tune)]),
    "mpc_ring_gemm_workspace_size": (c_size, [c_i64, c_i64, c_i64, c_int]),
    "mpc_ring_gemm": (c_int, [c_i64, c_i64, c_i64, c_vp, c_vp, c_vp, c_vp, c_int, c_vp, c_size,
                              c_vp]),
    "mpc_beaver_square": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_int, c_vp]),
    "mpc_ttp_square_pair": (c_int, [c_int, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp]),
    "mpc_ltz": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_u64, c_u64, c_vp]),
    "mpc_affine": (c_int, [c_int, c_i64, c_vp, c_vp, c_i64, c_u64, c_int, c_vp]),
    "mpc_private_relu_fused": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_vp]),
    "mpc_private_relu_fused_add": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_u64, c_u64, c_vp]),
    "mpc_private_max_fused": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_u64, c_u64, c_i64, c_vp]),
    "mpc_exp": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_vp]),
    "mpc_reciprocal": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_int, c_vp]),
    "mpc_sigmoid": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_vp]),
    "mpc_tanh": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_vp]),
    "mpc_erf": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_vp]),
    "mpc_inv_sqrt": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_vp]),
    "mpc_sqrt": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_vp]),
    "mpc_log": (c_int, [c_int, c_i64, c_vp, c_vp, c_u64, c_u64, c_int, c_int, c_int, c_vp]),
    "mpc_max_workspace_size": (c_size, [c_int, c_i64, c_i64]),
    "mpc_max_lastdim": (c_int, [c_int, c_i64, c_i64, c_vp, c_vp, c_vp, c_size, c_u64, c_u64,
                                c_vp]),
    "mpc_softmax_workspace_size": (c_size, [c_int, c_i64, c_i64]),
    "mpc_softmax": (c_int, [c_int, c_i64, c_i64, c_vp, c_vp, c_vp, c_size, c_u64, c_u64, c_int,
                            c_int, c_vp]),
    "mpc_truncate_nparty": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_int, c_vp]),
    "mpc_ttp_trunc_pairs": (c_int, [c_int, c_i64, c_u64, c_u64, c_vp, c_vp, c_vp]),
    "mpc_add": (c_int, [c_int, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "mpc_sub": (c_int, [c_int, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp]),
    "mpc_window_taps": (c_int, [c_int, _P(ConvDesc), c_vp, c_vp, c_vp]),
    "mpc_global_avgpool": (c_int, [c_int, c_i64, c_i64, c_vp, c_vp, c_vp]),
    "mpc_truncate": (c_int, [c_int, c_i64, c_vp, c_int, c_i64, c_vp]),
    "mpc_a2b": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_u64, c_u64, c_vp]),
    "mpc_private_relu": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                 c_u64, c_u64, c_vp]),
}

_lib = None


def load():
    """Load the shared library (once) and attach every signature."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_2109_00984_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
