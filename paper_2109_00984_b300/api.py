"""Python binding: argument marshalling from torch CUDA tensors to the C ABI.

Every function here only checks tensors, allocates outputs/workspaces with
torch (the caller's memory), and calls the entry point of the same name in
libmpcring.so on torch's current CUDA stream.  Ring words are carried in
torch.int64 (or torch.uint64) tensors: the bit pattern is the uint64 value.
No arithmetic of the protocol happens in Python.
"""
import ctypes

import torch

from . import _lib

PLAIN, LIMB, AUTO = 0, 1, 2
KS_GATES = 12
MAX_TRIPLE_BATCH = 8   # mpc_ring.h MPC_MAX_TRIPLE_BATCH
MAX_PARTIES = 8

MPC_OK = 0
STATUS_NAMES = {0: "MPC_OK", -1: "MPC_EINVAL", -2: "MPC_ERANGE", -3: "MPC_ENOMEM", -4: "MPC_ECUDA",
                -5: "MPC_ETIMEOUT", -6: "MPC_EUNSUPPORTED"}


class MPCError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _L():
    return _lib.load()


def _check(rc):
    if rc != MPC_OK:
        raise MPCError(rc, _L().mpc_last_error().decode(errors="replace"))


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


_WORD_DTYPES = (torch.int64, torch.uint64)


def _ptr(t, name="tensor", dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is None and t.dtype not in _WORD_DTYPES:
        raise ValueError(f"{name} must hold 64-bit ring words (int64/uint64), got {t.dtype}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _words(shape, device):
    return torch.empty(shape, dtype=torch.int64, device=device)


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def conv_desc(batch, c_in, h, w, c_out, kh, kw, stride_h=1, stride_w=1, pad_h=0, pad_w=0):
    return _lib.ConvDesc(batch, c_in, h, w, c_out, kh, kw, stride_h, stride_w, pad_h, pad_w)


def conv_out_hw(d):
    return ((d.h + 2 * d.pad_h - d.kh) // d.stride_h + 1,
            (d.w + 2 * d.pad_w - d.kw) // d.stride_w + 1)


# ---- status / counters ------------------------------------------------------------
def sync_status():
    """Synchronise the current stream and raise on a device-side error."""
    _check(_L().mpc_sync_status(_stream()))


def get_stats():
    s = _lib.Stats()
    _check(_L().mpc_get_stats(ctypes.byref(s)))
    return {f: int(getattr(s, f)) for f, _ in _lib.Stats._fields_}


def reset_stats():
    _check(_L().mpc_reset_stats())


def profile_enable(on=True):
    _check(_L().mpc_profile_enable(1 if on else 0))


def profile_reset():
    _check(_L().mpc_profile_reset())


def profile_read(kernel):
    """(launches, total_ms) of a timed kernel since the last profile_reset()."""
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(_L().mpc_profile_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def profile_busy(kernel):
    """Union of the device intervals of a timed kernel's launches (ms), over all streams."""
    ms = ctypes.c_double()
    _check(_L().mpc_profile_busy(kernel.encode(), ctypes.byref(ms)))
    return float(ms.value)


# ---- sharing / reveal ---------------------------------------------------------------
def ring_share(x, P, src, seed, op_id, frac_bits=16, out=None):
    """Encode float64 reals x (CUDA) and share among P parties -> [P, *x.shape]."""
    n = x.numel()
    out = _words((P,) + tuple(x.shape), x.device) if out is None else out
    _check(_L().mpc_ring_share(_ptr(x, "x", torch.float64), n, P, src, frac_bits, seed, op_id,
                               _ptr(out, "out"), _stream()))
    return out


def ring_share_encoded(x_ring, P, src, seed, op_id, out=None):
    n = x_ring.numel()
    out = _words((P,) + tuple(x_ring.shape), x_ring.device) if out is None else out
    _check(_L().mpc_ring_share_encoded(_ptr(x_ring, "x_ring"), n, P, src, seed, op_id,
                                       _ptr(out, "out"), _stream()))
    return out


def reveal(shares, frac_bits=16, ring=False, real=True):
    """Open [P, ...] shares; returns (ring or None, real or None)."""
    P = shares.shape[0]
    shape = tuple(shares.shape[1:])
    n = shares.numel() // P
    r = _words(shape, shares.device) if ring else None
    f = torch.empty(shape, dtype=torch.float64, device=shares.device) if real else None
    _check(_L().mpc_reveal(_ptr(shares, "shares"), P, n, frac_bits, _ptr(r),
                           _ptr(f, "real", torch.float64) if f is not None else None, _stream()))
    return r, f


# ---- dealer ---------------------------------------------------------------------------
def ttp_mul_triple(P, n, seed, op_id, device="cuda", out=None):
    A, B, C = out if out is not None else (_words((P, n), device) for _ in range(3))
    _check(_L().mpc_ttp_mul_triple(P, n, seed, op_id, _ptr(A), _ptr(B), _ptr(C), _stream()))
    return A, B, C


def ttp_matmul_triple(P, M, N, K, seed, op_id, algo=PLAIN, device="cuda", out=None, ws=None):
    A, B, C = out if out is not None else (_words((P, M, K), device), _words((P, K, N), device),
                                           _words((P, M, N), device))
    need = _L().mpc_matmul_triple_workspace_size(P, M, N, K, algo)
    ws = _ws(need, device) if ws is None else ws
    _check(_L().mpc_ttp_matmul_triple(P, M, N, K, seed, op_id, _ptr(A), _ptr(B), _ptr(C), algo,
                                      _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return A, B, C


def ttp_conv2d_triple(P, d, seed, op_id, algo=PLAIN, device="cuda", out=None, ws=None):
    ho, wo = conv_out_hw(d)
    if out is None:
        A = _words((P, d.batch, d.c_in, d.h, d.w), device)
        B = _words((P, d.c_out, d.c_in, d.kh, d.kw), device)
        C = _words((P, d.batch, d.c_out, ho, wo), device)
    else:
        A, B, C = out
    need = _L().mpc_conv2d_triple_workspace_size(P, ctypes.byref(d), algo)
    ws = _ws(need, device) if ws is None else ws
    _check(_L().mpc_ttp_conv2d_triple(P, ctypes.byref(d), seed, op_id, _ptr(A), _ptr(B), _ptr(C),
                                      algo, _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return A, B, C


def _desc_array(d, count):
    descs = [d] * count if isinstance(d, _lib.ConvDesc) else list(d)
    if len(descs) != count:
        raise ValueError(f"{len(descs)} descriptors for {count} triples")
    return (_lib.ConvDesc * count)(*descs), descs


def conv2d_triples_workspace_size(P, count, d, algo=PLAIN):
    """d: one descriptor for all `count` triples, or a list of count."""
    arr, _ = _desc_array(d, count)
    return int(_L().mpc_conv2d_triples_workspace_size(P, count, arr, algo))


def ttp_conv2d_triples(P, d, seed, op_ids, algo=PLAIN, device="cuda", outs=None, ws=None):
    """Convolution triples at each op id in `op_ids` (mpc_ttp_conv2d_triples):
    d is one descriptor for all of them or a list with one per op id (one
    output shape); outs: one (A, B, C) per op id, or None."""
    count = len(op_ids)
    arr, descs = _desc_array(d, count)
    if outs is None:
        outs = []
        for dj in descs:
            ho, wo = conv_out_hw(dj)
            outs.append((_words((P, dj.batch, dj.c_in, dj.h, dj.w), device),
                         _words((P, dj.c_out, dj.c_in, dj.kh, dj.kw), device),
                         _words((P, dj.batch, dj.c_out, ho, wo), device)))
    need = _L().mpc_conv2d_triples_workspace_size(P, count, arr, algo)
    ws = _ws(need, device) if ws is None else ws
    ids = (ctypes.c_uint64 * count)(*op_ids)
    ptrs = [(ctypes.c_void_p * count)(*[_ptr(t[i]) for t in outs]) for i in range(3)]
    _check(_L().mpc_ttp_conv2d_triples(P, count, arr, seed, ids, ptrs[0], ptrs[1], ptrs[2], algo,
                                       _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return outs


def ttp_and_triples(P, n, seed, op_id, gates=KS_GATES, device="cuda", out=None):
    T = _words((gates, 3, P, n), device) if out is None else out
    _check(_L().mpc_ttp_and_triples(P, n, gates, seed, op_id, _ptr(T), _stream()))
    return T


def ttp_b2a_bits(P, n, seed, op_id, device="cuda", out=None):
    if out is None:
        ra, rb = _words((P, n), device), _words((P, (n + 63) // 64), device)
    else:
        ra, rb = out
    _check(_L().mpc_ttp_b2a_bits(P, n, seed, op_id, _ptr(ra), _ptr(rb), _stream()))
    return ra, rb


# ---- online arithmetic -------------------------------------------------------------------
def beaver_mul(X, Y, A, B, C, trunc_bits=0, out=None, E_out=None, F_out=None):
    P = X.shape[0]
    n = X.numel() // P
    Z = torch.empty_like(X) if out is None else out
    _check(_L().mpc_beaver_mul(P, n, _ptr(X), _ptr(Y), _ptr(A), _ptr(B), _ptr(C), _ptr(Z),
                               _ptr(E_out), _ptr(F_out), trunc_bits, _stream()))
    return Z


def beaver_matmul(X, Y, A, B, C, algo=PLAIN, trunc_bits=0, out=None, ws=None):
    P, M, K = X.shape
    N = Y.shape[2]
    Z = _words((P, M, N), X.device) if out is None else out
    need = _L().mpc_matmul_workspace_size(P, M, N, K, algo)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_beaver_matmul(P, M, N, K, _ptr(X), _ptr(Y), _ptr(A), _ptr(B), _ptr(C),
                                  _ptr(Z), algo, trunc_bits, _ptr(ws, "ws", torch.uint8),
                                  ws.numel(), _stream()))
    return Z


def beaver_conv2d(X, W, A, B, C, d, algo=PLAIN, trunc_bits=0, out=None, ws=None):
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Z = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), algo)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_beaver_conv2d(P, ctypes.byref(d), _ptr(X), _ptr(W), _ptr(A), _ptr(B), _ptr(C),
                                  _ptr(Z), algo, trunc_bits, _ptr(ws, "ws", torch.uint8),
                                  ws.numel(), _stream()))
    return Z


def conv2d_prep_size(P, d):
    """Bytes of the prepared-plane buffer of a limb-engine Beaver convolution (0: unsupported)."""
    return _L().mpc_conv2d_prep_size(P, ctypes.byref(d))


def beaver_conv2d_prepare(W, A, B, d, out=None):
    """Input-independent half of a limb-engine Beaver convolution: opens F = W - B and cuts
    the digit planes of the weight side and of im2col(A_p) into a uint8 device buffer
    (returned), to be passed to beaver_conv2d_prepared / beaver_conv2d_relu_prepared with
    the same triple."""
    P = W.shape[0]
    need = conv2d_prep_size(P, d)
    if need == 0:
        raise MPCError(-6, "no prepared planes for this convolution shape")
    prep = torch.empty(need, dtype=torch.uint8, device=W.device) if out is None else out
    _check(_L().mpc_beaver_conv2d_prepare(P, ctypes.byref(d), _ptr(W), _ptr(A), _ptr(B),
                                          _ptr(prep, "prep", torch.uint8), prep.numel(),
                                          _stream()))
    return prep


def beaver_conv2d_prepared(X, A, C, prep, d, trunc_bits=0, out=None, ws=None):
    """Data-dependent half of a limb-engine Beaver convolution on prepared planes;
    equals beaver_conv2d(..., algo=LIMB)."""
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Z = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), LIMB)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_beaver_conv2d_prepared(P, ctypes.byref(d), _ptr(X), _ptr(A), _ptr(C),
                                           _ptr(prep, "prep", torch.uint8), prep.numel(), _ptr(Z),
                                           trunc_bits, _ptr(ws, "ws", torch.uint8), ws.numel(),
                                           _stream()))
    return Z


def conv2d_prep_products_size(P, d):
    return int(_L().mpc_conv2d_prep_products_size(P, ctypes.byref(d)))


def conv2d_prepare_products_workspace_size(P, d):
    return int(_L().mpc_conv2d_prepare_products_workspace_size(P, ctypes.byref(d)))


def beaver_conv2d_prepare_products(W, A, B, C, d, out=None, ws=None):
    """Input-independent half of a limb-engine Beaver convolution including each
    party's product: C'_p = C_p + A_p F (F = W - B opened) and the planes of
    G_p (G_0 = B_0 + F, G_p = B_p); returns the uint8 device buffer holding them."""
    P = W.shape[0]
    need = conv2d_prep_products_size(P, d)
    if need == 0:
        raise MPCError(-6, "no prepared products for this convolution shape")
    prep = torch.empty(need, dtype=torch.uint8, device=W.device) if out is None else out
    wneed = conv2d_prepare_products_workspace_size(P, d)
    ws = _ws(wneed, W.device) if ws is None else ws
    _check(_L().mpc_beaver_conv2d_prepare_products(
        P, ctypes.byref(d), _ptr(W), _ptr(A), _ptr(B), _ptr(C), _ptr(prep, "prep", torch.uint8),
        prep.numel(), _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return prep


def beaver_conv2d_prepared_products(X, A, prep, d, trunc_bits=0, out=None, ws=None):
    """Online half on prepared products (one operand pair per party); equals
    beaver_conv2d(..., algo=LIMB) with the same triple."""
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Z = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), LIMB)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_beaver_conv2d_prepared_products(
        P, ctypes.byref(d), _ptr(X), _ptr(A), _ptr(prep, "prep", torch.uint8), prep.numel(),
        _ptr(Z), trunc_bits, _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return Z


def beaver_conv2d_relu_prepared_products(X, A, prep, d, seed, relu_op, trunc_bits=0, out=None,
                                         ws=None):
    """beaver_conv2d_prepared_products then the fused private ReLU (two parties)."""
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Y = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), LIMB)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_beaver_conv2d_relu_prepared_products(
        P, ctypes.byref(d), _ptr(X), _ptr(A), _ptr(prep, "prep", torch.uint8), prep.numel(),
        _ptr(Y), trunc_bits, seed, relu_op, _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return Y


def beaver_conv2d_relu_prepared(X, A, C, prep, d, seed, relu_op, trunc_bits=0, out=None,
                                ws=None, add=None):
    """beaver_conv2d_prepared then the fused private ReLU (two parties); equals
    beaver_conv2d_relu(..., algo=LIMB).  With `add` (shares shaped like the
    output): the ReLU of the product plus add (a residual connection)."""
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Y = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), LIMB)
    ws = _ws(need, X.device) if ws is None else ws
    if add is None:
        _check(_L().mpc_beaver_conv2d_relu_prepared(
            P, ctypes.byref(d), _ptr(X), _ptr(A), _ptr(C), _ptr(prep, "prep", torch.uint8),
            prep.numel(), _ptr(Y), trunc_bits, seed, relu_op, _ptr(ws, "ws", torch.uint8),
            ws.numel(), _stream()))
    else:
        if add.numel() != Y.numel():
            raise ValueError("add must be shaped like the output")
        _check(_L().mpc_beaver_conv2d_relu_prepared_add(
            P, ctypes.byref(d), _ptr(X), _ptr(A), _ptr(C), _ptr(prep, "prep", torch.uint8),
            prep.numel(), _ptr(add, "add"), _ptr(Y), trunc_bits, seed, relu_op,
            _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return Y


def beaver_conv2d_relu(X, W, A, B, C, d, seed, relu_op, algo=PLAIN, trunc_bits=0, out=None,
                       ws=None, add=None):
    """Beaver convolution then the fused private ReLU (material at relu_op .. relu_op + 3),
    two parties; equals beaver_conv2d followed by private_relu_fused.  With `add`
    (shares shaped like the output): the ReLU of the product plus add."""
    P = X.shape[0]
    ho, wo = conv_out_hw(d)
    Y = _words((P, d.batch, d.c_out, ho, wo), X.device) if out is None else out
    need = _L().mpc_conv2d_workspace_size(P, ctypes.byref(d), algo)
    ws = _ws(need, X.device) if ws is None else ws
    if add is None:
        _check(_L().mpc_beaver_conv2d_relu(P, ctypes.byref(d), _ptr(X), _ptr(W), _ptr(A), _ptr(B),
                                           _ptr(C), _ptr(Y), algo, trunc_bits, seed, relu_op,
                                           _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    else:
        if add.numel() != Y.numel():
            raise ValueError("add must be shaped like the output")
        _check(_L().mpc_beaver_conv2d_relu_add(
            P, ctypes.byref(d), _ptr(X), _ptr(W), _ptr(A), _ptr(B), _ptr(C), _ptr(add, "add"),
            _ptr(Y), algo, trunc_bits, seed, relu_op, _ptr(ws, "ws", torch.uint8), ws.numel(),
            _stream()))
    return Y


def conv2d_workspace_size(P, d, algo=PLAIN):
    return int(_L().mpc_conv2d_workspace_size(P, ctypes.byref(d), algo))


def conv2d_triple_workspace_size(P, d, algo=PLAIN):
    return int(_L().mpc_conv2d_triple_workspace_size(P, ctypes.byref(d), algo))


def matmul_workspace_size(P, M, N, K, algo=PLAIN):
    return int(_L().mpc_matmul_workspace_size(P, M, N, K, algo))


def ring_gemm(A, B, C=None, algo=PLAIN, out=None, ws=None):
    M, K = A.shape
    N = B.shape[1]
    Z = _words((M, N), A.device) if out is None else out
    need = _L().mpc_ring_gemm_workspace_size(M, N, K, algo)
    ws = _ws(need, A.device) if ws is None else ws
    _check(_L().mpc_ring_gemm(M, N, K, _ptr(A), _ptr(B), _ptr(C), _ptr(Z), algo,
                              _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))
    return Z


def ring_gemm_workspace_size(M, N, K, algo=PLAIN):
    return int(_L().mpc_ring_gemm_workspace_size(M, N, K, algo))


# ---- batched Beaver matmul -----------------------------------------------------------
class BatchedMatmul:
    """Marshalled argument set of mpc_beaver_matmul_batched for a fixed batch.

    products: list of (X, Y, A, B, C, Z) CUDA tensors, X [P, M, K], Y [P, K, N],
    A/B/C the Beaver triple, Z the output [P, M, N].  The descriptor array is
    built once, so repeated calls (and a CUDA graph capture of a call) do no
    per-product Python work.
    """

    def __init__(self, products, algo=AUTO, trunc_bits=16, tune=None):
        self.P = products[0][0].shape[0]
        self.count = len(products)
        self.descs = (_lib.MatmulDesc * self.count)()
        for i, (X, Y, A, B, C, Z) in enumerate(products):
            P, M, K = X.shape
            N = Y.shape[2]
            assert P == self.P and Z.shape == (P, M, N)
            self.descs[i] = _lib.MatmulDesc(M, N, K, *[ctypes.c_void_p(t.data_ptr()) for t in (
                X, Y, A, B, C, Z)])
            for t in (X, Y, A, B, C, Z):
                _ptr(t)
        self.products = products          # keep the tensors alive
        self.algo = algo
        self.trunc_bits = trunc_bits
        self.tune = tune if tune is not None else default_tune()
        self.ws = None

    def workspace_size(self):
        return int(_L().mpc_matmul_batched_workspace_size(self.P, self.count, self.descs, self.algo,
                                                          ctypes.byref(self.tune)))

    def ensure_workspace(self, device="cuda"):
        need = self.workspace_size()
        if self.ws is None or self.ws.numel() < need:
            self.ws = _ws(need, device)
        return self.ws

    def __call__(self):
        ws = self.ensure_workspace(self.products[0][0].device)
        _check(_L().mpc_beaver_matmul_batched(self.P, self.count, self.descs, self.algo,
                                              ctypes.byref(self.tune), self.trunc_bits,
                                              _ptr(ws, "ws", torch.uint8), ws.numel(), _stream()))

    def autotune(self, ws_bytes=None):
        """Pick the limb threshold by timing the call (synchronises; writes Z)."""
        dev = self.products[0][0].device
        if ws_bytes is None:
            everything = _lib.Tune(1.0, 0, 0)    # the largest plan: every product on limb
            ws_bytes = int(_L().mpc_matmul_batched_workspace_size(
                self.P, self.count, self.descs, LIMB, ctypes.byref(everything)))
        ws = _ws(ws_bytes, dev)
        out = _lib.Tune()
        _check(_L().mpc_autotune_batched(self.P, self.count, self.descs, self.trunc_bits,
                                         _ptr(ws, "ws", torch.uint8), ws.numel(), _stream(),
                                         ctypes.byref(out)))
        self.tune = out
        self.algo = AUTO
        self.ws = None
        return out


def default_tune():
    t = _lib.Tune()
    _check(_L().mpc_tune_default(ctypes.byref(t)))
    return t


def beaver_matmul_batched(products, algo=AUTO, trunc_bits=16, tune=None):
    """One call of mpc_beaver_matmul_batched over `products` (see BatchedMatmul)."""
    bm = BatchedMatmul(products, algo, trunc_bits, tune)
    bm()
    return bm


def truncate(shares, frac_bits=16, divisor=0):
    """In place on [P, ...] shares; returns shares."""
    P = shares.shape[0]
    _check(_L().mpc_truncate(P, shares.numel() // P, _ptr(shares), frac_bits, divisor, _stream()))
    return shares


def ttp_trunc_pairs(P, n, seed, op_id, device="cuda", out=None):
    """Alg. 1 dealer material: (r [P, n], theta_r [P, n])."""
    r, th = out if out is not None else (_words((P, n), device), _words((P, n), device))
    _check(_L().mpc_ttp_trunc_pairs(P, n, seed, op_id, _ptr(r), _ptr(th), _stream()))
    return r, th


def truncate_nparty(shares, r, theta_r, frac_bits=16):
    """Alg. 1 truncation in place on [P, ...] shares; returns shares."""
    P = shares.shape[0]
    _check(_L().mpc_truncate_nparty(P, shares.numel() // P, _ptr(shares), _ptr(r), _ptr(theta_r),
                                    frac_bits, _stream()))
    return shares


# ---- local share operations ------------------------------------------------------
def _party_view(t, P):
    """(pointer, words per party, party stride) of a [P, ...] tensor or party-strided view."""
    n = t[0].numel()
    if not t[0].is_contiguous():
        raise ValueError("each party's slice must be contiguous")
    stride = t.stride(0) if P > 1 else n
    return ctypes.c_void_p(t.data_ptr()), n, stride


def add(X, Y, out=None):
    """Z = X + Y share by share (party-strided views allowed)."""
    P = X.shape[0]
    Z = torch.empty_like(X) if out is None else out
    xp, n, xs = _party_view(X, P)
    yp, _, ys = _party_view(Y, P)
    zp, _, zs = _party_view(Z, P)
    _check(_L().mpc_add(P, n, xp, xs, yp, ys, zp, zs, _stream()))
    return Z


def sub(X, Y, out=None):
    """Z = X - Y share by share (party-strided views allowed)."""
    P = X.shape[0]
    Z = torch.empty_like(X) if out is None else out
    xp, n, xs = _party_view(X, P)
    yp, _, ys = _party_view(Y, P)
    zp, _, zs = _party_view(Z, P)
    _check(_L().mpc_sub(P, n, xp, xs, yp, ys, zp, zs, _stream()))
    return Z


def window_taps(X, k, stride, pad, out=None):
    """X [P, N, C, H, W] -> taps [k*k, P, N, C, Ho, Wo] (zero padded)."""
    P, N, C, H, W = X.shape
    d = conv_desc(N, C, H, W, C, k, k, stride, stride, pad, pad)
    ho, wo = conv_out_hw(d)
    T = _words((k * k, P, N, C, ho, wo), X.device) if out is None else out
    _check(_L().mpc_window_taps(P, ctypes.byref(d), _ptr(X), _ptr(T), _stream()))
    return T


def global_avgpool(X, out=None):
    """X [P, N, C, H, W] -> [P, N, C]: local sum, then floor division by H*W."""
    P, N, C, H, W = X.shape
    out = _words((P, N, C), X.device) if out is None else out
    _check(_L().mpc_global_avgpool(P, N * C, H * W, _ptr(X), _ptr(out), _stream()))
    return out


# ---- binary / comparison -----------------------------------------------------------------
def a2b(X, and_triples, seed, op_id, out=None):
    P = X.shape[0]
    n = X.numel() // P
    out = torch.empty_like(X) if out is None else out
    _check(_L().mpc_a2b(P, n, _ptr(X), _ptr(out), _ptr(and_triples), seed, op_id, _stream()))
    return out


def private_relu(X, and_triples, r_arith, r_bin, mul_triple, seed, op_id, out=None):
    """mul_triple: the elementwise triple (A, B, C), each [P, n]-shaped (or a [3, P, n]
    tensor, whose three slices are passed as they lie)."""
    P = X.shape[0]
    n = X.numel() // P
    MA, MB, MC = mul_triple[0], mul_triple[1], mul_triple[2]
    out = torch.empty_like(X) if out is None else out
    _check(_L().mpc_private_relu(P, n, _ptr(X), _ptr(out), _ptr(and_triples), _ptr(r_arith),
                                 _ptr(r_bin), _ptr(MA, "mul A"), _ptr(MB, "mul B"),
                                 _ptr(MC, "mul C"), seed, op_id, _stream()))
    return out


def private_relu_fused(X, seed, op_id, out=None, add=None):
    """ReLU with the dealer fused in: material from op ids op_id .. op_id + 3 (P = 2).
    With `add` (shares shaped like X): the ReLU of X + add, the addition folded in."""
    P = X.shape[0]
    n = X.numel() // P
    out = torch.empty_like(X) if out is None else out
    if add is None:
        _check(_L().mpc_private_relu_fused(P, n, _ptr(X), _ptr(out), seed, op_id, _stream()))
    else:
        if add.numel() != X.numel():
            raise ValueError("add must have X's number of words")
        _check(_L().mpc_private_relu_fused_add(P, n, _ptr(X), _ptr(add, "add"), _ptr(out), seed,
                                               op_id, _stream()))
    return out


def private_max_fused(A, B, seed, op_id, elem_offset=0, out=None):
    """max(A, B) = B + ReLU(A - B) on two-party shares (P = 2), the ReLU's material
    that of elements elem_offset .. of a batched comparison at op ids op_id .. + 3."""
    P = A.shape[0]
    n = A.numel() // P
    if B.numel() != A.numel():
        raise ValueError("A and B must have the same number of words")
    out = torch.empty_like(A) if out is None else out
    _check(_L().mpc_private_max_fused(P, n, _ptr(A), _ptr(B, "B"), _ptr(out), seed, op_id,
                                      elem_offset, _stream()))
    return out


# ---- square, comparators, multiplexing ----------------------------------------------
def ttp_square_pair(P, n, seed, op_id, device="cuda", out=None):
    A, B = out if out is not None else (_words((P, n), device), _words((P, n), device))
    _check(_L().mpc_ttp_square_pair(P, n, seed, op_id, _ptr(A), _ptr(B), _stream()))
    return A, B


def beaver_square(X, A, B, trunc_bits=0, out=None):
    P = X.shape[0]
    Z = torch.empty_like(X) if out is None else out
    _check(_L().mpc_beaver_square(P, X.numel() // P, _ptr(X), _ptr(A), _ptr(B), _ptr(Z), trunc_bits,
                                  _stream()))
    return Z


def affine(X, scale, offset=0, trunc_bits=0, out=None):
    """Z_p = scale * X_p (+ offset on party 0), optional two-party truncation."""
    P = X.shape[0]
    Z = torch.empty_like(X) if out is None else out
    _check(_L().mpc_affine(P, X.numel() // P, _ptr(X), _ptr(Z), int(scale),
                           int(offset) % (1 << 64), trunc_bits, _stream()))
    return Z


def ltz(X, seed, op_id, out=None):
    """[x < 0] as unscaled 0/1 shares; material at op_id, op_id + 1, masks at op_id + 3."""
    P = X.shape[0]
    n = X.numel() // P
    T = ttp_and_triples(P, n, seed, op_id, gates=KS_GATES * (P - 1), device=X.device)
    ra, rb = ttp_b2a_bits(P, n, seed, op_id + 1, device=X.device)
    out = torch.empty_like(X) if out is None else out
    _check(_L().mpc_ltz(P, n, _ptr(X), _ptr(out), _ptr(T), _ptr(ra), _ptr(rb), seed, op_id + 3,
                        _stream()))
    return out


def lt(X, Y, seed, op_id):
    return ltz(sub(X, Y), seed, op_id)


def gt(X, Y, seed, op_id):
    return ltz(sub(Y, X), seed, op_id)


def ge(X, Y, seed, op_id):
    return affine(lt(X, Y, seed, op_id), -1, 1)


def le(X, Y, seed, op_id):
    return affine(gt(X, Y, seed, op_id), -1, 1)


def eq(X, Y, seed, op_id):
    """[x <= y] - [x < y]; the two comparisons use op_id and op_id + 10."""
    return sub(le(X, Y, seed, op_id), lt(X, Y, seed, op_id + 10))


def ne(X, Y, seed, op_id):
    return affine(eq(X, Y, seed, op_id), -1, 1)


def mux(C, X, Y, seed, op_id):
    """[c ? x : y] = [c] ([x] - [y]) + [y] with the elementwise triple at op_id."""
    P = C.shape[0]
    n = C.numel() // P
    A, B, T = ttp_mul_triple(P, n, seed, op_id, device=C.device)
    prod = beaver_mul(C, sub(X, Y), A.view(C.shape), B.view(C.shape), T.view(C.shape))
    return add(prod, Y)


# ---- function approximations (App. D.2), two parties, one fused launch each ----------
# Step k of a function draws its dealer material at op id op_id + 10 k.
EXP_ITERS = 8
NR_ITERS = 10
ERF_TERMS = 8
LOG_ITERS = 3
LOG_ORDER = 8


def _elementwise(fn, X, out, *args):
    P = X.shape[0]
    n = X.numel() // P
    out = torch.empty_like(X) if out is None else out
    _check(fn(P, n, _ptr(X), _ptr(out), *args, _stream()))
    return out


def exp(X, seed, op_id, iters=EXP_ITERS, out=None):
    """exp by the limit approximation (1 + x / 2^iters)^(2^iters)."""
    return _elementwise(_L().mpc_exp, X, out, seed, op_id, iters)


def reciprocal(X, seed, op_id, all_positive=False, exp_iters=EXP_ITERS, nr_iters=NR_ITERS,
               out=None):
    """1/x by Newton-Raphson from 3 exp(0.5 - x) + 0.003; sgn(x) / |x| unless all_positive."""
    return _elementwise(_L().mpc_reciprocal, X, out, seed, op_id, int(bool(all_positive)),
                        exp_iters, nr_iters)


def sigmoid(X, seed, op_id, exp_iters=EXP_ITERS, nr_iters=NR_ITERS, out=None):
    return _elementwise(_L().mpc_sigmoid, X, out, seed, op_id, exp_iters, nr_iters)


def tanh(X, seed, op_id, exp_iters=EXP_ITERS, nr_iters=NR_ITERS, out=None):
    return _elementwise(_L().mpc_tanh, X, out, seed, op_id, exp_iters, nr_iters)


def erf(X, seed, op_id, terms=ERF_TERMS, out=None):
    return _elementwise(_L().mpc_erf, X, out, seed, op_id, terms)


def inv_sqrt(X, seed, op_id, exp_iters=EXP_ITERS, nr_iters=NR_ITERS, out=None):
    return _elementwise(_L().mpc_inv_sqrt, X, out, seed, op_id, exp_iters, nr_iters)


def sqrt(X, seed, op_id, exp_iters=EXP_ITERS, nr_iters=NR_ITERS, out=None):
    return _elementwise(_L().mpc_sqrt, X, out, seed, op_id, exp_iters, nr_iters)


def log(X, seed, op_id, exp_iters=EXP_ITERS, iters=LOG_ITERS, order=LOG_ORDER, out=None):
    return _elementwise(_L().mpc_log, X, out, seed, op_id, exp_iters, iters, order)


def max_lastdim(X, seed, op_id, out=None, ws=None):
    """Maximum over the last axis of shares [2, ..., m] -> [2, ...] (exact, ReLU tree)."""
    P, m = X.shape[0], X.shape[-1]
    rows = X.numel() // (P * m)
    out = torch.empty(X.shape[:-1], dtype=torch.int64, device=X.device) if out is None else out
    need = _L().mpc_max_workspace_size(P, rows, m)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_max_lastdim(P, rows, m, _ptr(X), _ptr(out), _ptr(ws, "ws", torch.uint8),
                                ws.numel(), seed, op_id, _stream()))
    return out


def softmax(X, seed, op_id, exp_iters=EXP_ITERS, nr_iters=NR_ITERS, out=None, ws=None):
    """Softmax over the last axis of shares [2, ..., m]."""
    P, m = X.shape[0], X.shape[-1]
    rows = X.numel() // (P * m)
    out = torch.empty_like(X) if out is None else out
    need = _L().mpc_softmax_workspace_size(P, rows, m)
    ws = _ws(need, X.device) if ws is None else ws
    _check(_L().mpc_softmax(P, rows, m, _ptr(X), _ptr(out), _ptr(ws, "ws", torch.uint8), ws.numel(),
                            seed, op_id, exp_iters, nr_iters, _stream()))
    return out
