"""Pins for the oracle's CNN layer operations and the ResNet-18-shaped forward.

Max pooling is checked against a brute-force window maximum (zero padding) on
revealed values, global average pooling against floor division of the exact
sum (within the two-party truncation's one-unit slack), and the whole private
forward against the independent float64 forward (NMSE < 4e-4, §6.1).
"""
import numpy as np

import synth
from oracle import fixed, resnet, sharing


def _share(v):
    return sharing.share(np.asarray(v, dtype=np.int64).view(np.uint64), 2, 0, 1, 9)


def test_window_taps_brute_force(rng):
    x = rng.integers(0, 2 ** 64, (2, 1, 2, 5, 6), dtype=np.uint64)
    taps = resnet.window_taps(x, 3, 2, 1)
    Ho, Wo = 3, 3
    for t in range(9):
        r, s = divmod(t, 3)
        for i in range(Ho):
            for j in range(Wo):
                y, xx = i * 2 + r - 1, j * 2 + s - 1
                want = x[:, :, :, y, xx] if (0 <= y < 5 and 0 <= xx < 6) else 0
                assert np.array_equal(taps[t][:, :, :, i, j], np.broadcast_to(want, taps[t][:, :, :, i, j].shape))


def test_maxpool_tree_is_window_max(rng):
    v = rng.integers(-(1 << 40), 1 << 40, (1, 3, 7, 8))
    X = _share(v)
    got = sharing.reveal(resnet.maxpool_shares(X, 3, 2, 1, [11, 21, 31, 41], 1)).view(np.int64)
    vp = np.zeros((1, 3, 9, 10), dtype=np.int64)
    vp[:, :, 1:8, 1:9] = v
    want = np.zeros(got.shape, dtype=np.int64)
    for i in range(got.shape[2]):
        for j in range(got.shape[3]):
            want[:, :, i, j] = vp[:, :, 2 * i:2 * i + 3, 2 * j:2 * j + 3].max(axis=(2, 3))
    assert np.array_equal(got, want)


def test_global_avgpool_floor(rng):
    v = rng.integers(-(1 << 40), 1 << 40, (1, 4, 7, 7))
    got = sharing.reveal(resnet.global_avgpool_shares(_share(v))).view(np.int64)
    exact = np.array([[int(s) // 49 for s in row] for row in v.reshape(1, 4, 49).sum(-1)])
    assert set(np.unique(got - exact).tolist()) <= {-1, 0}


def test_private_resnet18_small_matches_float64():
    x = synth.resnet_input(batch=2, hw=32)
    W = synth.resnet_weights()
    sched = synth.resnet_schedule()
    Wsh = resnet.share_resnet_weights(W, synth.RESNET18, sched)
    out = resnet.private_resnet18(x, Wsh, synth.RESNET18, sched)
    ref = resnet.plaintext_resnet18(x, W, synth.RESNET18)
    assert out.shape == ref.shape == (2, 1000)
    nmse = float(((out - ref) ** 2).sum() / (ref ** 2).sum())
    assert nmse < 4e-4
