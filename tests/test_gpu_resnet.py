"""Private ResNet-18-shaped inference on the GPU against the oracle, bit-exact.

Layer operations (window taps, local add/sub, global average pooling, the
max-pool tree) are compared one by one; the reduced network (32 x 32 inputs,
batch 2) is compared on every output share; the full configuration bench.py
times (batch 8 of 224 x 224) is compared on image 0, which the oracle computes
as a batch of one: every PRG stream is indexed by flat element position and
the data are batch-major, so image 0's material is the prefix of each stream.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev, dev_f64, host  # noqa: E402

import synth  # noqa: E402
from oracle import resnet as oresnet  # noqa: E402
from oracle import sharing  # noqa: E402


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def test_window_taps(mpc, rng):
    X = rng.integers(0, 2 ** 64, (2, 2, 3, 9, 7), dtype=np.uint64)
    got = host(mpc.window_taps(dev(X), 3, 2, 1))
    assert np.array_equal(got, oresnet.window_taps(X, 3, 2, 1))


def test_add_sub_party_strided(mpc, rng):
    X = rng.integers(0, 2 ** 64, (2, 3, 1001), dtype=np.uint64)
    Y = rng.integers(0, 2 ** 64, (2, 1001), dtype=np.uint64)
    dX, dY = dev(X), dev(Y)
    with np.errstate(over="ignore"):
        assert np.array_equal(host(mpc.add(dX[:, 1], dY)), X[:, 1] + Y)
        out = torch.empty((2, 3, 1001), dtype=torch.int64, device="cuda")
        mpc.sub(dX[:, 2], dY, out=out[:, 0])
        assert np.array_equal(host(out)[:, 0], X[:, 2] - Y)


def test_global_avgpool(mpc, rng):
    X = rng.integers(0, 2 ** 64, (2, 3, 5, 7, 7), dtype=np.uint64)
    got = host(mpc.global_avgpool(dev(X)))
    assert np.array_equal(got, oresnet.global_avgpool_shares(X))


@pytest.mark.parametrize("shape", [
    (2, 4, 11, 10),   # 120 outputs: the fused comparison per pair (a multiple of 4)
    (2, 3, 9, 9),     # 75 outputs: the batched sub / ReLU / add fallback
])
def test_maxpool_tree(mpc, rng, shape):
    from paper_2109_00984_b300.resnet import PrivateResNet18
    v = rng.integers(0, 1 << 40, shape).astype(np.int64)
    X = sharing.share(v.view(np.uint64), 2, 0, 1, 3)
    net = PrivateResNet18({}, [], synth.resnet_schedule(), fused_relu=False)
    got = host(net.maxpool(dev(X), 3, 2, 1, [101, 111, 121, 131]))
    net_f = PrivateResNet18({}, [], synth.resnet_schedule(), fused_relu=True)
    assert np.array_equal(host(net_f.maxpool(dev(X), 3, 2, 1, [101, 111, 121, 131])), got)
    ref = oresnet.maxpool_shares(X, 3, 2, 1, [101, 111, 121, 131], 1)
    assert np.array_equal(got, ref)


def _gpu_forward(mpc, x, algo=None, fused=True, prepared=False):
    from paper_2109_00984_b300.resnet import PrivateResNet18
    W = synth.resnet_weights()
    sched = synth.resnet_schedule()
    net = PrivateResNet18(W, synth.RESNET18, sched, algo=mpc.AUTO if algo is None else algo,
                          fused_relu=fused, prepare_weights=prepared)
    Y = net.forward(dev_f64(x), sched)
    real = net.reveal(Y)
    torch.cuda.synchronize()
    return host(Y), real.cpu().numpy()


def _oracle_forward(x):
    W = synth.resnet_weights()
    sched = synth.resnet_schedule()
    Wsh = oresnet.share_resnet_weights(W, synth.RESNET18, sched)
    real, shares = oresnet.private_resnet18(x, Wsh, synth.RESNET18, sched, return_shares=True)
    return shares, real, W


@pytest.mark.parametrize("engine,fused", [("plain", False), ("auto", True)])
def test_small_resnet_bit_exact(mpc, engine, fused):
    x = synth.resnet_input(batch=2, hw=32)
    got, got_real = _gpu_forward(mpc, x, mpc.PLAIN if engine == "plain" else mpc.AUTO, fused)
    ref, ref_real, _ = _oracle_forward(x)
    assert np.array_equal(got, ref)
    assert np.array_equal(got_real, ref_real)


def test_small_resnet_prepared_bit_exact(mpc):
    """The dealer also prepares every convolution's input-independent half; the
    online phase runs the prepared convolutions: the same words."""
    x = synth.resnet_input(batch=2, hw=32)
    got, got_real = _gpu_forward(mpc, x, prepared=True)
    ref, ref_real, _ = _oracle_forward(x)
    assert np.array_equal(got, ref)
    assert np.array_equal(got_real, ref_real)


@pytest.mark.slow
def test_full_resnet_image0_bit_exact(mpc):
    """Batch 8 x 224 x 224 (the bench configuration); image 0 against the oracle."""
    x = synth.resnet_input(batch=8, hw=224)
    got, got_real = _gpu_forward(mpc, x, prepared=True)   # the bench's configuration
    ref, ref_real, W = _oracle_forward(x[:1])
    assert np.array_equal(got[:, :1], ref)
    plain = oresnet.plaintext_resnet18(x, W, synth.RESNET18)
    nmse = float(((got_real - plain) ** 2).sum() / (plain ** 2).sum())
    assert nmse < 4e-4


@pytest.mark.parametrize("prepared", [False, True])
def test_small_resnet_graph_replay_bit_exact(mpc, prepared):
    """The bench's timed path: a captured forward + reveal, replayed, equals the oracle."""
    from paper_2109_00984_b300.resnet import PrivateResNet18
    x = synth.resnet_input(batch=2, hw=32)
    sched = synth.resnet_schedule(step=4)
    net = PrivateResNet18(synth.resnet_weights(), synth.RESNET18, sched, algo=mpc.AUTO,
                          prepare_weights=prepared)
    xd = dev_f64(x)
    net.reveal(net.forward(xd, synth.resnet_schedule(step=9)))   # warm-up sizes the workspaces
    (g, out), = net.capture(xd, [sched])
    g.replay()
    torch.cuda.synchronize()
    W = synth.resnet_weights()
    Wsh = oresnet.share_resnet_weights(W, synth.RESNET18, sched)
    ref_real, _ = oresnet.private_resnet18(x, Wsh, synth.RESNET18, sched, return_shares=True)
    assert np.array_equal(out.cpu().numpy(), ref_real)
