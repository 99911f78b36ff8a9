"""The private speech-shaped conv stack on the GPU against the oracle, bit-exact.

The reduced stack (3 layers, ragged lengths) checks every share of every
layer's output; the full stack (80 -> 256 channels, 1600 frames, 7 layers: the
workload bench.py times, in the same launch configuration) checks every share
of the final output against the oracle's complete private forward, and the
decoded output against float64 within the paper's NMSE bound (§6.1: < 4e-4).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from gpu_util import dev_f64, host  # noqa: E402

import synth  # noqa: E402
from oracle import nets  # noqa: E402


@pytest.fixture(scope="module")
def mpc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2109_00984_b300 as m
    return m


def _run(mpc, x, ws, strides, pads, algo, step=0, fused=True):
    from paper_2109_00984_b300.nets import PrivateConv1dStack
    sched = synth.speech_schedule(len(ws), step=step)
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=x.shape[0], algo=algo,
                             weight_ops=sched["weight_op"], seed=sched["seed"], fused_relu=fused)
    Y = net.forward(dev_f64(x), sched)
    real = net.reveal(Y)
    torch.cuda.synchronize()
    return host(Y), real.cpu().numpy(), sched


def _oracle(x, ws, strides, pads, sched):
    Wsh = nets.share_weights(ws, sched)
    return nets.private_conv1d_stack(x, Wsh, strides, pads, sched, return_shares=True)


@pytest.mark.parametrize("step,fused", [(0, False), (3, False), (0, True)])
def test_small_stack_bit_exact(mpc, step, fused):
    x, ws, strides, pads = synth.speech_small()
    got_shares, got_real, sched = _run(mpc, x, ws, strides, pads, mpc.PLAIN, step, fused)
    ref_real, ref_shares = _oracle(x, ws, strides, pads, sched)
    assert np.array_equal(got_shares.reshape(ref_shares.shape), ref_shares)
    assert np.array_equal(got_real.reshape(ref_real.shape), ref_real)


@pytest.fixture(scope="module")
def full_oracle():
    x, ws, strides, pads = synth.speech_stack()
    sched = synth.speech_schedule(len(ws))
    ref_real, ref_shares = _oracle(x, ws, strides, pads, sched)
    plain = nets.plaintext_conv1d_stack(x, ws, strides, pads)
    return ref_shares, plain


@pytest.mark.slow
@pytest.mark.parametrize("engine", ["plain", "auto"])
def test_full_speech_stack_bit_exact(mpc, full_oracle, engine):
    """Full stack; "auto" is bench.py's configuration (limb engine, fused-dealer ReLU)."""
    x, ws, strides, pads = synth.speech_stack()
    algo = mpc.PLAIN if engine == "plain" else mpc.AUTO
    got_shares, got_real, sched = _run(mpc, x, ws, strides, pads, algo, fused=(engine == "auto"))
    ref_shares, plain = full_oracle
    assert np.array_equal(got_shares.reshape(ref_shares.shape), ref_shares)
    nmse = float(((got_real.reshape(plain.shape) - plain) ** 2).sum() / (plain ** 2).sum())
    assert nmse < 4e-4


def _captured(mpc, x, ws, strides, pads, algo, schedules):
    """Forward + reveal captured as CUDA graphs (the bench's timed path), replayed."""
    from paper_2109_00984_b300.nets import PrivateConv1dStack
    s0 = schedules[0]
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=x.shape[0], algo=algo,
                             weight_ops=s0["weight_op"], seed=s0["seed"])
    xd = dev_f64(x)
    graphs = net.capture(xd, schedules)
    results = []
    for g, out in graphs:
        g.replay()
        torch.cuda.synchronize()
        results.append((host(net.bufs[-1]["Y"]), out.cpu().numpy()))
    return results


def test_small_stack_graph_replay_bit_exact(mpc):
    """Each replayed graph equals the oracle's forward for its own schedule."""
    x, ws, strides, pads = synth.speech_small()
    scheds = [synth.speech_schedule(len(ws), step=s) for s in (5, 6)]
    for (got_shares, got_real), sched in zip(_captured(mpc, x, ws, strides, pads, mpc.AUTO, scheds),
                                             scheds):
        ref_real, ref_shares = _oracle(x, ws, strides, pads, sched)
        assert np.array_equal(got_shares.reshape(ref_shares.shape), ref_shares)
        assert np.array_equal(got_real.reshape(ref_real.shape), ref_real)


@pytest.mark.slow
def test_full_speech_stack_graph_replay_bit_exact(mpc, full_oracle):
    """The bench's timed path: graph replay of the full stack, limb engine, fused ReLU."""
    x, ws, strides, pads = synth.speech_stack()
    sched = synth.speech_schedule(len(ws))
    (got_shares, got_real), = _captured(mpc, x, ws, strides, pads, mpc.AUTO, [sched])
    ref_shares, plain = full_oracle
    assert np.array_equal(got_shares.reshape(ref_shares.shape), ref_shares)
    nmse = float(((got_real.reshape(plain.shape) - plain) ** 2).sum() / (plain ** 2).sum())
    assert nmse < 4e-4


@pytest.mark.parametrize("prepared", [False, True])
def test_small_stack_pipelined_bit_exact(mpc, prepared):
    """Software-pipelined steps (online phase of batch i on the triples dealt
    during step i - 1), as graph replays and eagerly: every output equals the
    oracle's forward for its own schedule.  prepared: the dealer also runs each
    convolution's input-independent half (beaver_conv2d_prepare)."""
    from paper_2109_00984_b300.nets import PrivateConv1dStack
    x, ws, strides, pads = synth.speech_small()
    scheds = [synth.speech_schedule(len(ws), step=s) for s in (11, 12, 13, 14)]
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=x.shape[0], algo=mpc.AUTO,
                             weight_ops=scheds[0]["weight_op"], seed=scheds[0]["seed"],
                             prepare_weights=prepared)
    assert net.prepared == prepared
    xd = dev_f64(x)
    refs = [_oracle(x, ws, strides, pads, s) for s in scheds[:3]]
    graphs = net.capture_pipelined(xd, scheds[:3], scheds[1:])
    net.deal(scheds[0], 0, join=True)
    for (g, out), (ref_real, ref_shares) in zip(graphs, refs):
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(net.bufs[-1]["Y"]).reshape(ref_shares.shape), ref_shares)
        assert np.array_equal(out.cpu().numpy().reshape(ref_real.shape), ref_real)
    net.deal(scheds[0], 0)     # eager steps wait on the dealer's events instead
    for i, (ref_real, ref_shares) in enumerate(refs):
        Y = net.forward_pipelined(xd, scheds[i], i % 2, scheds[i + 1])
        real = net.reveal(Y)
        torch.cuda.synchronize()
        assert np.array_equal(host(Y).reshape(ref_shares.shape), ref_shares)
        assert np.array_equal(real.cpu().numpy().reshape(ref_real.shape), ref_real)


def test_small_stack_pipelined_two_input_buffers(mpc):
    """Pipelined graphs reading alternating input buffers (graph i reads
    buffer i % 2, so the next input can be uploaded while a step runs): each
    step's output equals the oracle's forward on that step's own input."""
    from paper_2109_00984_b300.nets import PrivateConv1dStack
    x, ws, strides, pads = synth.speech_small()
    x2 = x[..., ::-1].copy()   # a second, different input of the same shape
    scheds = [synth.speech_schedule(len(ws), step=s) for s in (21, 22, 23, 24)]
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=x.shape[0], algo=mpc.AUTO,
                             weight_ops=scheds[0]["weight_op"], seed=scheds[0]["seed"])
    inputs = [x, x2, x]
    bufs = [dev_f64(x), dev_f64(x2)]
    refs = [_oracle(inp, ws, strides, pads, s) for inp, s in zip(inputs, scheds[:3])]
    graphs = net.capture_pipelined(bufs, scheds[:3], scheds[1:])
    net.deal(scheds[0], 0, join=True)
    for (g, out), (ref_real, ref_shares) in zip(graphs, refs):
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(host(net.bufs[-1]["Y"]).reshape(ref_shares.shape), ref_shares)
        assert np.array_equal(out.cpu().numpy().reshape(ref_real.shape), ref_real)


@pytest.mark.slow
@pytest.mark.parametrize("products", [False, True])
def test_full_speech_stack_prepared_bit_exact(mpc, full_oracle, products):
    """The full stack with the convolutions' input-independent half on the
    dealer (the bench's schedule; with `products` also each party's A_p F, the
    online-latency schedule) gives the oracle's shares."""
    from paper_2109_00984_b300.nets import PrivateConv1dStack
    x, ws, strides, pads = synth.speech_stack()
    sched = synth.speech_schedule(len(ws))
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=x.shape[0], algo=mpc.AUTO,
                             weight_ops=sched["weight_op"], seed=sched["seed"],
                             prepare_weights=True, prepare_products=products)
    assert net.prepared and net.prep_products == products
    Y = net.forward(dev_f64(x), sched)
    torch.cuda.synchronize()
    ref_shares, plain = full_oracle
    assert np.array_equal(host(Y).reshape(ref_shares.shape), ref_shares)
