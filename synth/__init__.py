"""Seeded synthetic workloads shared by the tests, the oracle checks and bench.py.

This module holds input recipes and protocol schedules only (shapes, seeds,
random reals, op_id numbering); it contains none of the protocol's arithmetic
and imports neither the oracle nor the CUDA package.

The paper's datasets (Yelp, LibriSpeech, ImageNet) and trained weights are not
available, so every workload is a synthetic stand-in with the benchmark's
shapes and stated value distributions.
"""
import numpy as np

PROTOCOL_SEED = 1
FRAC_BITS = 16


# --- small matmul / elementwise case ---------------------------------------
def small_case():
    """X 64x128, Y 128x32 and two 4096-vectors, uniform[-4, 4], rng seed 0."""
    rng = np.random.default_rng(0)
    X = rng.uniform(-4, 4, (64, 128))
    Y = rng.uniform(-4, 4, (128, 32))
    xe = rng.uniform(-4, 4, 4096)
    ye = rng.uniform(-4, 4, 4096)
    return X, Y, xe, ye


SMALL_SCHEDULE = dict(seed=PROTOCOL_SEED, x_op=1, y_op=2, xe_op=3, ye_op=4,
                      matmul_triple_op=10, mul_triple_op=11)


# --- speech-shaped 1-D conv stack ------------------------------------------
SPEECH_LAYERS = [  # (Cin, Cout, k, stride, pad)
    (80, 256, 11, 2, 5),
] + [(256, 256, 7, 1, 3)] * 6
SPEECH_FRAMES = 1600


def speech_stack(batch=1, frames=SPEECH_FRAMES, layers=SPEECH_LAYERS, seed=0):
    """Input (batch, 80, frames) ~ N(0, 1), then weights ~ N(0, 0.05) per layer."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((batch, layers[0][0], frames))
    ws = [rng.normal(0.0, 0.05, (co, ci, k)) for (ci, co, k, _, _) in layers]
    strides = [s for (_, _, _, s, _) in layers]
    pads = [p for (_, _, _, _, p) in layers]
    return x, ws, strides, pads


def speech_schedule(n_layers=len(SPEECH_LAYERS), step=0):
    """op_id numbering for one private forward of the conv stack.

    ``step`` offsets every id so that successive forwards draw fresh material.
    """
    base = 1 + 1000 * step
    return dict(
        seed=PROTOCOL_SEED,
        input_op=base,
        weight_op=[900000 + l for l in range(n_layers)],
        layers=[dict(conv=base + 10 * l + 1, **{"and": base + 10 * l + 2},
                     b2a=base + 10 * l + 3, mul=base + 10 * l + 4, relu=base + 10 * l + 5)
                for l in range(n_layers)],
    )


def speech_small(seed=0):
    """A reduced stack with the same structure (ragged sizes) for fast parity."""
    layers = [(5, 24, 11, 2, 5), (24, 24, 7, 1, 3), (24, 24, 7, 1, 3)]
    return speech_stack(batch=1, frames=203, layers=layers, seed=seed)


# --- ring GEMM sweep ---------------------------------------------------------
GEMM_SIZES = (1024, 2048, 4096, 8192)


def uniform_ring(shape, seed=0):
    """uint64 words uniform over Z/2^64."""
    return np.random.default_rng(seed).integers(0, 2 ** 64, size=shape, dtype=np.uint64,
                                                endpoint=False)


# --- batched uneven matmuls --------------------------------------------------
def batched_dims(count=512, lo=32, hi=2048, seed=2):
    """(M, N, K) triples log-uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), (count, 3)))).astype(np.int64)


# --- ResNet-18-shaped CNN --------------------------------------------------
# Layer list: ("conv", name, cin, cout, k, stride, pad) | ("relu", name) |
# ("maxpool", name, k, stride, pad) | ("block", name, cin, cout, stride) |
# ("avgpool", name) | ("fc", name, cin, cout).  BatchNorm at its initial
# statistics is the identity up to its epsilon and is folded away; no biases.
RESNET18 = (
    [("conv", "conv1", 3, 64, 7, 2, 3), ("relu", "relu1"), ("maxpool", "maxpool", 3, 2, 1)]
    + [("block", f"layer{i}.{j}", cin if j == 0 else cout, cout, s if j == 0 else 1)
       for i, (cin, cout, s) in enumerate([(64, 64, 1), (64, 128, 2), (128, 256, 2),
                                            (256, 512, 2)], start=1) for j in range(2)]
    + [("avgpool", "avgpool"), ("fc", "fc", 512, 1000)]
)


def resnet_weights(seed=0, classes=1000):
    """He-initialised weights, std = sqrt(2 / fan_in), in RESNET18 order.

    Returns a dict name -> float64 array: convs (cout, cin, k, k), the FC weight
    transposed to (cin, classes) so that logits = x @ W.
    """
    rng = np.random.default_rng(seed + 1)
    W = {}

    def conv(name, cin, cout, k):
        W[name] = rng.normal(0.0, np.sqrt(2.0 / (cin * k * k)), (cout, cin, k, k))

    for layer in RESNET18:
        kind = layer[0]
        if kind == "conv":
            conv(layer[1], layer[2], layer[3], layer[4])
        elif kind == "block":
            _, name, cin, cout, s = layer
            conv(name + ".conv1", cin, cout, 3)
            conv(name + ".conv2", cout, cout, 3)
            if s != 1 or cin != cout:
                conv(name + ".down", cin, cout, 1)
        elif kind == "fc":
            W[layer[1]] = rng.normal(0.0, np.sqrt(2.0 / layer[2]), (layer[2], classes))
    return W


def resnet_input(batch=8, hw=224, seed=0):
    """Images (batch, 3, hw, hw) ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal((batch, 3, hw, hw))


def resnet_schedule(step=0):
    """op_ids for one private forward: 10 ids per layer op, in forward order."""
    base = 2_000_000 + 100_000 * step
    ops = {}
    k = 0

    def take(name):
        nonlocal k
        ops[name] = base + 10 * k
        k += 1

    take("input")
    for layer in RESNET18:
        kind, name = layer[0], layer[1]
        if kind in ("conv", "relu", "fc"):
            take(name)
        elif kind == "maxpool":
            for lvl in range(4):
                take(f"{name}.{lvl}")
        elif kind == "block":
            for part in ("conv1", "relu1", "conv2", "down", "relu2"):
                take(f"{name}.{part}")
    return dict(seed=PROTOCOL_SEED, ops=ops, weight_base=3_000_000)
