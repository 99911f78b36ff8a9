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
