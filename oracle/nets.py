"""Compositions of the protocol: a private 1-D conv stack and its plaintext twin.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A speech-shaped stack (§6.2 evaluates Wav2Letter, a stack of 1-D convolutions
with ReLU): each layer is a Beaver convolution (§5.2 "Linear functions"),
local truncation by 2^16 (App. D.1.1) and a private ReLU (§5.2
"Comparators").  The weights are secret-shared by party 1 (the model owner),
the input by party 0 (the data owner).  No bias.

``schedule`` fixes which (seed, op_id) every sharing and every piece of dealer
material uses; it is plain data supplied by the caller, so that the oracle and
the device pipeline consume identical randomness.
"""
import numpy as np

from . import binary, dealer, fixed, ring, sharing, truncation
from .beaver import beaver_conv2d
from .transcript import _maybe


def plaintext_conv1d_stack(x, weights, strides, pads):
    """float64 reference: x (1, Cin, L); ReLU(conv1d(...)) per layer."""
    h = np.asarray(x, dtype=np.float64)
    for w, s, pd in zip(weights, strides, pads):
        Cout, Cin, k = w.shape
        Lo = (h.shape[2] + 2 * pd - k) // s + 1
        hp = np.zeros((h.shape[0], Cin, h.shape[2] + 2 * pd))
        hp[:, :, pd:pd + h.shape[2]] = h
        out = np.zeros((h.shape[0], Cout, Lo))
        for t in range(k):
            win = hp[:, :, t:t + s * (Lo - 1) + 1:s]
            out += np.einsum("oc,ncl->nol", w[:, :, t], win)
        h = np.maximum(out, 0.0)
    return h


def share_weights(weights, schedule, frac_bits=16):
    """Party 1 shares every layer's encoded weights: list of [2][Cout][Cin][k]."""
    seed = schedule["seed"]
    return [sharing.share(fixed.encode(w, frac_bits), 2, 1, seed, schedule["weight_op"][l])
            for l, w in enumerate(weights)]


def private_conv1d_layer(X, W, stride, pad, ops, seed, frac_bits=16, tr=None):
    """One layer on shares X [2][1][Cin][L], W [2][Cout][Cin][k]."""
    tr = _maybe(tr)
    P = X.shape[0]
    x4 = X[:, :, :, None, :]          # (P, N, Cin, 1, L)
    w4 = W[:, :, :, None, :]          # (P, Cout, Cin, 1, k)
    A, B, C = dealer.conv2d_triple(P, x4.shape[1:], w4.shape[1:], stride, 0, seed,
                                   ops["conv"], pad_w=pad)
    Z = beaver_conv2d(x4, w4, A, B, C, stride, 0, pad_w=pad, tr=tr)
    Z = truncation.truncate(Z, frac_bits)
    Zf = Z.reshape(P, -1)
    n = Zf.shape[1]
    T = dealer.and_triples(P, n, binary.KS_GATES, seed, ops["and"])
    r_arith, r_bin = dealer.b2a_bits(P, n, seed, ops["b2a"])
    mt = dealer.mul_triple(P, n, seed, ops["mul"])
    Y = binary.private_relu(Zf, T, r_arith, r_bin, mt, seed, ops["relu"], tr)
    return Y.reshape(Z.shape[0], Z.shape[1], Z.shape[2], Z.shape[4])


def private_conv1d_stack(x, Wsh, strides, pads, schedule, frac_bits=16, tr=None,
                         return_shares=False):
    """Private forward of the stack; returns decoded float64 output (and shares)."""
    seed = schedule["seed"]
    X = sharing.share(fixed.encode(x, frac_bits), 2, 0, seed, schedule["input_op"])
    for l, (W, s, pd) in enumerate(zip(Wsh, strides, pads)):
        X = private_conv1d_layer(X, W, s, pd, schedule["layers"][l], seed, frac_bits, tr)
    out = fixed.decode(sharing.reveal(X), frac_bits)
    return (out, X) if return_shares else out


def ring_conv1d_reference(x_ring, w_ring, stride, pad):
    """Ring conv1d (for sampled checks); x (N, Cin, L), w (Cout, Cin, k)."""
    return ring.conv1d(x_ring, w_ring, stride=stride, pad=pad)
