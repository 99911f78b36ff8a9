"""Private inference of a ResNet-18-shaped CNN, and its float64 twin.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Layer operations (the paper evaluates ResNet-18 inference, §6.3; the function
table of App. B lists the operations):
  * convolution and linear layer: Beaver product with the bilinear f (App.
    D.1.1), then truncation by 2^16;
  * ReLU: the comparator-based private ReLU (§5.2);
  * residual connection: private addition, local (§5.2 "Private addition");
  * 3x3 / stride-2 max pooling: a tree of pairwise maxima,
    max(a, b) = b + ReLU(a - b) (App. D.1.4 builds max from comparisons); the
    nine window taps (zero padding: inputs are ReLU outputs, so a 0 pad never
    wins over a real element) are reduced level by level, 9 -> 5 -> 3 -> 2 ->
    1, all pairs of one level sharing one ReLU call laid out [P][pair][n];
  * global average pooling: a local sum over the window, then division by the
    public window size as two-party truncation (floor of each share, App.
    D.1.1);
  * BatchNorm at its initial statistics is the identity (up to its epsilon)
    and is folded away.
Readings: the residual add precedes the block's second ReLU (the standard
BasicBlock); no biases.
"""
import numpy as np

from . import binary, dealer, fixed, sharing, truncation
from .beaver import beaver_conv2d, beaver_matmul

U64 = np.uint64


# ---- float64 twin -------------------------------------------------------------------
def _conv_f64(x, w, stride, pad):
    N, Cin, H, W = x.shape
    Cout, _, k, _ = w.shape
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (W + 2 * pad - k) // stride + 1
    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad))
    xp[:, :, pad:pad + H, pad:pad + W] = x
    out = np.zeros((N, Cout, Ho, Wo))
    for r in range(k):
        for s in range(k):
            win = xp[:, :, r:r + stride * (Ho - 1) + 1:stride, s:s + stride * (Wo - 1) + 1:stride]
            out += np.einsum("oc,nchw->nohw", w[:, :, r, s], win)
    return out


def _maxpool_f64(x, k, stride, pad):
    N, C, H, W = x.shape
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (W + 2 * pad - k) // stride + 1
    xp = np.full((N, C, H + 2 * pad, W + 2 * pad), -np.inf)
    xp[:, :, pad:pad + H, pad:pad + W] = x
    out = np.full((N, C, Ho, Wo), -np.inf)
    for r in range(k):
        for s in range(k):
            out = np.maximum(out, xp[:, :, r:r + stride * (Ho - 1) + 1:stride,
                                     s:s + stride * (Wo - 1) + 1:stride])
    return out


def plaintext_resnet18(x, W, layers):
    h = np.asarray(x, dtype=np.float64)
    for layer in layers:
        kind = layer[0]
        if kind == "conv":
            h = _conv_f64(h, W[layer[1]], layer[5], layer[6])
        elif kind == "relu":
            h = np.maximum(h, 0.0)
        elif kind == "maxpool":
            h = _maxpool_f64(h, layer[2], layer[3], layer[4])
        elif kind == "block":
            _, name, cin, cout, s = layer
            y = np.maximum(_conv_f64(h, W[name + ".conv1"], s, 1), 0.0)
            y = _conv_f64(y, W[name + ".conv2"], 1, 1)
            sc = _conv_f64(h, W[name + ".down"], s, 0) if (s != 1 or cin != cout) else h
            h = np.maximum(y + sc, 0.0)
        elif kind == "avgpool":
            h = h.mean(axis=(2, 3))
        elif kind == "fc":
            h = h @ W[layer[1]]
    return h


# ---- private operations ----------------------------------------------------------------
def relu_shares(X, op, seed, tr=None):
    """Private ReLU of shares X [P, ...] with material drawn at op .. op+3."""
    P = X.shape[0]
    flat = X.reshape(P, -1)
    n = flat.shape[1]
    T = dealer.and_triples(P, n, binary.KS_GATES, seed, op)
    ra, rb = dealer.b2a_bits(P, n, seed, op + 1)
    mt = dealer.mul_triple(P, n, seed, op + 2)
    return binary.private_relu(flat, T, ra, rb, mt, seed, op + 3, tr).reshape(X.shape)


def conv_shares(X, Wsh, stride, pad, op, seed, frac_bits=16, tr=None):
    P = X.shape[0]
    A, B, C = dealer.conv2d_triple(P, X.shape[1:], Wsh.shape[1:], stride, pad, seed, op)
    return truncation.truncate(beaver_conv2d(X, Wsh, A, B, C, stride, pad, tr=tr), frac_bits)


def window_taps(X, k, stride, pad):
    """[k*k][P][N][C][Ho][Wo] window taps of shares X [P][N][C][H][W], zero padded."""
    P, N, C, H, W = X.shape
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (W + 2 * pad - k) // stride + 1
    xp = np.zeros((P, N, C, H + 2 * pad, W + 2 * pad), dtype=U64)
    xp[..., pad:pad + H, pad:pad + W] = X
    taps = [xp[..., r:r + stride * (Ho - 1) + 1:stride, s:s + stride * (Wo - 1) + 1:stride]
            for r in range(k) for s in range(k)]
    return np.stack(taps)


def maxpool_shares(X, k, stride, pad, ops, seed, tr=None):
    """Tree of max(a, b) = b + ReLU(a - b) over the k*k taps (one ReLU call per level)."""
    taps = window_taps(X, k, stride, pad)
    P = X.shape[0]
    shape = taps.shape[1:]
    vals = [t.reshape(P, -1) for t in taps]
    n = vals[0].shape[1]
    level = 0
    with np.errstate(over="ignore"):
        while len(vals) > 1:
            npairs = len(vals) // 2
            D = np.stack([vals[2 * i] - vals[2 * i + 1] for i in range(npairs)], axis=1)  # [P][pair][n]
            R = relu_shares(D.reshape(P, npairs * n), ops[level], seed, tr).reshape(P, npairs, n)
            new = [vals[2 * i + 1] + R[:, i] for i in range(npairs)]
            if len(vals) % 2:
                new.append(vals[-1])
            vals = new
            level += 1
    return vals[0].reshape(shape)


def global_avgpool_shares(X):
    """Local sum over H x W, then floor division of each share by H * W."""
    P, N, C, H, W = X.shape
    with np.errstate(over="ignore"):
        S = X.reshape(P, N, C, H * W).sum(axis=-1, dtype=U64)
    return truncation.truncate(S, 0, divisor=H * W)


def share_resnet_weights(W, layers, schedule, frac_bits=16):
    """The model owner (party 1) shares every weight; op_id weight_base + index."""
    seed = schedule["seed"]
    out = {}
    for i, name in enumerate(sorted(W)):
        out[name] = sharing.share(fixed.encode(W[name], frac_bits), 2, 1, seed,
                                  schedule["weight_base"] + i)
    return out


def private_resnet18(x, Wsh, layers, schedule, frac_bits=16, tr=None, return_shares=False):
    seed, ops = schedule["seed"], schedule["ops"]
    X = sharing.share(fixed.encode(x, frac_bits), 2, 0, seed, ops["input"])
    for layer in layers:
        kind, name = layer[0], layer[1]
        if kind == "conv":
            X = conv_shares(X, Wsh[name], layer[5], layer[6], ops[name], seed, frac_bits, tr)
        elif kind == "relu":
            X = relu_shares(X, ops[name], seed, tr)
        elif kind == "maxpool":
            X = maxpool_shares(X, layer[2], layer[3], layer[4],
                               [ops[f"{name}.{l}"] for l in range(4)], seed, tr)
        elif kind == "block":
            _, name, cin, cout, s = layer
            Y = conv_shares(X, Wsh[name + ".conv1"], s, 1, ops[name + ".conv1"], seed, frac_bits, tr)
            Y = relu_shares(Y, ops[name + ".relu1"], seed, tr)
            Y = conv_shares(Y, Wsh[name + ".conv2"], 1, 1, ops[name + ".conv2"], seed, frac_bits, tr)
            if s != 1 or cin != cout:
                S = conv_shares(X, Wsh[name + ".down"], s, 0, ops[name + ".down"], seed,
                                frac_bits, tr)
            else:
                S = X
            with np.errstate(over="ignore"):
                X = relu_shares(Y + S, ops[name + ".relu2"], seed, tr)
        elif kind == "avgpool":
            X = global_avgpool_shares(X)
        elif kind == "fc":
            P, N, Cin = X.shape
            Cout = Wsh[name].shape[2]
            A, B, C = dealer.matmul_triple(P, N, Cout, Cin, seed, ops[name])
            X = truncation.truncate(beaver_matmul(X, Wsh[name], A, B, C, tr), frac_bits)
    out = fixed.decode(sharing.reveal(X), frac_bits)
    return (out, X) if return_shares else out
