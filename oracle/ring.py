"""Bilinear maps over the ring Z/2^64 (uint64 wraparound).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

§5.2 "Linear functions": matrix products and convolutions are the bilinear f of
the Beaver identity (App. D.1.1, "holds for any linear function f").  These are
the plain definitions: numpy's uint64 matmul wraps mod 2^64, and the
convolution is the direct sliding-window sum (cross-correlation, as in deep
learning frameworks), zero padding, no bias, groups = 1, dilation = 1.
"""
import numpy as np

U64 = np.uint64


def matmul(a, b):
    """(M, K) x (K, N) -> (M, N) over Z/2^64."""
    a = np.asarray(a, dtype=U64)
    b = np.asarray(b, dtype=U64)
    with np.errstate(over="ignore"):
        return np.matmul(a, b)


def conv2d_out_hw(H, W, kh, kw, stride, pad):
    return (H + 2 * pad - kh) // stride + 1, (W + 2 * pad - kw) // stride + 1


def conv2d(x, w, stride=1, pad=0, pad_w=None):
    """x: (N, Cin, H, W), w: (Cout, Cin, kh, kw) -> (N, Cout, Ho, Wo) over Z/2^64.

    out[n, co, i, j] = sum_{ci, r, s} w[co, ci, r, s] * xpad[n, ci, i*stride + r, j*stride + s]
    ``pad`` pads H, ``pad_w`` (default ``pad``) pads W.
    """
    x = np.asarray(x, dtype=U64)
    w = np.asarray(w, dtype=U64)
    if pad_w is None:
        pad_w = pad
    N, Cin, H, W = x.shape
    Cout, Cin2, kh, kw = w.shape
    assert Cin == Cin2
    Ho = (H + 2 * pad - kh) // stride + 1
    Wo = (W + 2 * pad_w - kw) // stride + 1
    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad_w), dtype=U64)
    xp[:, :, pad:pad + H, pad_w:pad_w + W] = x
    out = np.zeros((N, Cout, Ho, Wo), dtype=U64)
    with np.errstate(over="ignore"):
        for r in range(kh):
            for s in range(kw):
                win = xp[:, :, r:r + stride * (Ho - 1) + 1:stride, s:s + stride * (Wo - 1) + 1:stride]
                # (Cout, Cin) x (N, Cin, Ho*Wo) -> (N, Cout, Ho*Wo)
                tap = np.matmul(w[:, :, r, s][None], win.reshape(N, Cin, Ho * Wo))
                out += tap.reshape(N, Cout, Ho, Wo)
    return out


def conv1d(x, w, stride=1, pad=0):
    """x: (N, Cin, L), w: (Cout, Cin, k) -> (N, Cout, Lo); conv2d with H = 1."""
    y = conv2d(np.asarray(x)[:, :, None, :], np.asarray(w)[:, :, None, :], stride=stride,
               pad=0, pad_w=pad)
    return y[:, :, 0, :]
