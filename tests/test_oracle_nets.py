"""End-to-end sanity of the oracle's private conv stack against float64.

§6.1 reports a normalised MSE below 4e-4 against the plaintext model; here the
stack is the reduced speech-shaped stack, checked against a float64 numpy
forward written independently of the ring code.
"""
import numpy as np

import synth
from oracle import nets


def test_private_small_speech_stack_matches_float64():
    x, ws, strides, pads = synth.speech_small()
    sched = synth.speech_schedule(len(ws))
    Wsh = nets.share_weights(ws, sched)
    out = nets.private_conv1d_stack(x, Wsh, strides, pads, sched)
    ref = nets.plaintext_conv1d_stack(x, ws, strides, pads)
    assert out.shape == ref.shape
    nmse = float(((out - ref) ** 2).sum() / (ref ** 2).sum())
    assert nmse < 4e-4
    # Per-element: a few fixed-point ulps per layer.
    assert np.max(np.abs(out - ref)) < 1e-2
