"""Benchmark: private inference of the speech-shaped conv stack on B300.

One step = one full private forward of one sample (2 parties, batch 1, input
80 x 1600 frames, Conv1d 80->256 k11 s2 then 6x Conv1d 256->256 k7, ring
Z/2^64 with 2^16 fixed point): share the input, and for each layer let the
dealer produce the convolution triple and the ReLU material, run the Beaver
convolution with fused truncation and the fused private ReLU; then reveal.
Every step of the hot path runs in libmpcring.so kernels.

Prints ONE JSON line (rank 0).  Under torchrun (N > 1) every rank runs its own
replica on its own sample: no data-path collective, weak scaling.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--algo plain|limb|auto]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "Beaver ring-GEMM TOPS (Z/2^64, bit-exact): i8-limb TC vs plain CUDA-core; samples/s"
WORKLOAD = ("speech-shaped private conv stack: 2 parties, batch 1, input 80x1600, "
            "Conv1d 80->256 k11 s2 + 6x Conv1d 256->256 k7 (pad k//2), each Beaver conv + "
            "truncation 2^16 + private ReLU (A2B/Kogge-Stone/B2A), Z/2^64, dealer in the step")
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic of the limb GEMM per launch, averaged over the 8 launches of one
# speech step (7 online GEMMs of two pairs for two parties, and one launch for
# the dealer's seven one-pair products), from an ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum on the current kernel; and the
# digit-plane bytes those launches must read (785.5 MB per step: 16 bytes per
# operand word).
LIMB_GEMM_DRAM_BYTES_PER_LAUNCH = 110.9e6
LIMB_GEMM_PLANE_BYTES_PER_LAUNCH = 98.2e6
# ncu sm__pipe_tensor_cycles_active (% of elapsed cycles) of the same kernel in
# one capture each: an online speech-layer launch, and the 4096^3 ring GEMM.
LIMB_GEMM_TENSOR_ACTIVE_SPEECH = 64.4
# ... and time-weighted over the eight limb GEMM launches of one speech forward.
LIMB_GEMM_TENSOR_ACTIVE_SPEECH_STEP = 62.6
LIMB_GEMM_TENSOR_ACTIVE_4096 = 80.7
REF_FRAMES = 160          # oracle sample: the whole stack on 1/10 of the frames


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--algo", default="auto", choices=["plain", "limb", "auto"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements of the default line (GEMM sweep, "
                         "HBM-bound kernels, ResNet-18, batched products)")
    ap.add_argument("--workload", default="speech",
                    choices=["speech", "gemm", "batched", "resnet", "approx", "elementwise"],
                    help="speech: the private conv stack (default); gemm: ring GEMM sweep; "
                         "batched: 512 uneven Beaver matmuls; elementwise: the HBM-bound "
                         "kernels at n = 2^20 .. 2^26")
    ap.add_argument("--sizes", default="1024,2048,4096,8192")
    ap.add_argument("--elem-log2", default="20,22,24,26",
                    help="elementwise workload: log2 of the element counts")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="batched workload: number of products (the first of the seed-2 draw)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def job_time(local_s, world, device=None):
    """Max over ranks of a per-rank duration (the slowest replica sets the pace).

    Replicas share nothing on the data path; this reduction is the only
    collective, used for timing only.
    """
    if world <= 1:
        return float(local_s)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, slowest_s):
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return world * units_per_rank / slowest_s


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mpc_bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- reference arm
def oracle_forward(frames, step):
    """One private forward of the stack through the CPU oracle on `frames` frames."""
    from oracle import nets
    x, ws, strides, pads = synth.speech_stack(frames=frames)
    sched = synth.speech_schedule(len(ws), step=step)
    Wsh = nets.share_weights(ws, sched)
    return nets.private_conv1d_stack(x, Wsh, strides, pads, sched)


def _oracle_sample_seconds(step):
    t = time.perf_counter()
    oracle_forward(REF_FRAMES, step)
    return time.perf_counter() - t


ORACLE_MAX_PROCS = 32

# Oracle samples of the other workloads, bounded (a few seconds each).
ORACLE_GEMM_N = 1024          # ring GEMM n^3: numpy uint64 matmul, not BLAS
ORACLE_RESNET_HW = (56, 112)  # one image at two resolutions, extrapolated to 224


def _oracle_gemm_rows(args):
    """Rows [r0, r1) of the n^3 ring GEMM through the oracle; compute seconds."""
    from oracle import ring
    n, r0, r1 = args
    rng = np.random.default_rng(0)
    a = rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64)
    b = rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64)
    t = time.perf_counter()
    ring.matmul(a[r0:r1], b)
    return time.perf_counter() - t


def oracle_gemm_measure(n=ORACLE_GEMM_N, all_cores=True):
    """The oracle's ring GEMM at n^3 on one core and as row blocks over all cores."""
    dt = _oracle_gemm_rows((n, 0, n))
    out = {"value": 2 * n ** 3 / dt / 1e12, "unit": "ring TOPS", "cores": 1, "kind": "oracle",
           "sample": f"M = N = K = {n} ({dt:.1f} s; numpy uint64 matmul, single-threaded); "
                     f"at 4096^3 / 8192^3 this rate gives {64 * dt:.0f} / {512 * dt:.0f} s "
                     f"(extrapolated by n^3; the per-MAC rate falls as n grows)",
           "extrapolated_s": {"4096": 64 * dt, "8192": 512 * dt}}
    if all_cores:
        import multiprocessing
        procs = max(1, min(os.cpu_count() or 1, ORACLE_MAX_PROCS))
        bounds = [(n, i * n // procs, (i + 1) * n // procs) for i in range(procs)]
        with multiprocessing.get_context("spawn").Pool(procs) as pool:
            secs = pool.map(_oracle_gemm_rows, bounds)
        out["all_cores"] = {"value": 2 * n ** 3 / max(secs) / 1e12, "unit": "ring TOPS",
                            "cores": procs,
                            "sample": f"row blocks of the same GEMM, one process each "
                                      f"(slowest {max(secs):.2f} s)"}
    return out


def oracle_resnet_measure(hws=ORACLE_RESNET_HW):
    """One image of the private ResNet-18-shaped inference through the oracle at two
    input resolutions (dealer included, weights shared beforehand); the time is
    fitted as a + b * pixels and extrapolated to 224 x 224."""
    from oracle import resnet as oresnet
    sched = synth.resnet_schedule()
    Wsh = oresnet.share_resnet_weights(synth.resnet_weights(), synth.RESNET18, sched)
    secs = []
    for hw in hws:
        x = synth.resnet_input(batch=1, hw=hw)
        t = time.perf_counter()
        oresnet.private_resnet18(x, Wsh, synth.RESNET18, sched)
        secs.append(time.perf_counter() - t)
    (h0, h1), (t0, t1) = hws, secs
    slope = (t1 - t0) / (h1 * h1 - h0 * h0)
    t224 = t1 + slope * (224 * 224 - h1 * h1)
    return {"value": 1 / t224, "unit": "images/s", "cores": 1, "kind": "oracle",
            "extrapolated": True,
            "sample": f"one image at {h0}x{h0} ({t0:.1f} s) and {h1}x{h1} ({t1:.1f} s), "
                      f"time fitted linearly in pixels and extrapolated to 224x224 "
                      f"({t224:.1f} s per image); numpy uint64 single-threaded"}


def cpu_baseline_measure(steps=1, all_cores=True):
    t = time.perf_counter()
    for s in range(steps):
        oracle_forward(REF_FRAMES, s)
    dt = (time.perf_counter() - t) / steps
    scale = REF_FRAMES / synth.SPEECH_FRAMES
    out = {"value": scale / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
           "sample": f"whole 7-layer private forward on the first {REF_FRAMES} of "
                     f"{synth.SPEECH_FRAMES} frames ({dt:.1f} s), samples/s scaled by "
                     f"{REF_FRAMES}/{synth.SPEECH_FRAMES}; numpy uint64 single-threaded"}
    if all_cores:
        # The same sample in one spawned process per core (capped), all at once:
        # throughput = processes x sample / the slowest process's compute time.
        import multiprocessing
        n = max(1, min(os.cpu_count() or 1, ORACLE_MAX_PROCS))
        with multiprocessing.get_context("spawn").Pool(n) as pool:
            secs = pool.map(_oracle_sample_seconds, range(n))
        out["all_cores"] = {"value": n * scale / max(secs), "unit": "samples/s", "cores": n,
                            "sample": f"{n} concurrent processes, one sample each "
                                      f"(slowest {max(secs):.1f} s)"}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for w in range(args.warmup):
        oracle_forward(REF_FRAMES, 100 + w)
    t = time.perf_counter()
    for s in range(args.steps):
        oracle_forward(REF_FRAMES, s)
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    value = (REF_FRAMES / synth.SPEECH_FRAMES) / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parties": 2, "batch": 1,
                       "reference": "CPU oracle (numpy uint64), bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step: whole stack on {REF_FRAMES} of "
                                       f"{synth.SPEECH_FRAMES} frames, scaled"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def layer_macs(net):
    """Ring multiply-adds per forward in the conv GEMMs (dealer + all parties)."""
    tot = 0
    for d in net.descs:
        M, K = d.c_out, d.c_in * d.kh * d.kw
        N = d.batch * ((d.w + 2 * d.pad_w - d.kw) // d.stride_w + 1)
        tot += (1 + 2 * net.P) * M * N * K      # dealer c = a.b, then P parties x 2 pairs
    return tot


def relu_bytes_per_elem(P=2):
    # x, y shares; 12 AND gates x (a, b, c) x P words; [r] P words + <r> P bits;
    # elementwise triple 3 x P words.
    return 8 * P + 8 * 12 * 3 * P + 8 * P + P / 8.0 + 8 * 3 * P + 8 * P


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2109_00984_b300 as mpc
    from paper_2109_00984_b300.nets import PrivateConv1dStack

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    algo = {"plain": mpc.PLAIN, "limb": mpc.LIMB, "auto": mpc.AUTO}[args.algo]

    x, ws, strides, pads = synth.speech_stack(seed=rank)
    sched0 = synth.speech_schedule(len(ws), step=0)
    # The dealer also prepares each convolution's input-independent half (F = W - B
    # opened, the weight-side and im2col(A_p) digit planes) for the online phase.
    net = PrivateConv1dStack(ws, strides, pads, x.shape[2], batch=1, algo=algo,
                             weight_ops=sched0["weight_op"], seed=sched0["seed"], device=dev,
                             prepare_weights=True)
    x_dev = torch.from_numpy(x).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(i, inp):
        Y = net.forward(inp, synth.speech_schedule(len(ws), step=i))
        return net.reveal(Y)

    for w in range(args.warmup):
        step(1000 + w, x_dev)
    torch.cuda.synchronize()

    # Each timed step replays a CUDA graph captured with that step's own
    # schedule (one host call per step, every kernel re-run).  The steps are
    # software-pipelined as an MPC offline phase runs: step i runs the online
    # phase of batch i on the triples dealt during step i - 1 while its dealer
    # deals the triples of batch i + 1 on the other stream -- one forward's
    # dealing and one forward's online phase per step.  The launch count is
    # taken from the library's counter while the timed steps are captured.
    scheds = [synth.speech_schedule(len(ws), step=i) for i in range(args.steps + 1)]
    mpc.reset_stats()
    graphs = net.capture_pipelined(x_dev, scheds[:-1], scheds[1:])
    stats = mpc.get_stats()
    net.deal(scheds[0], 0, join=True)
    for g, _ in graphs:          # first launches upload the graphs (untimed)
        g.replay()
    net.deal(scheds[0], 0, join=True)   # step 0's triples again: replays consume their own
    torch.cuda.synchronize()

    # ---- device-timed region: K steps, L2 flushed between steps ----------
    # The headline pass runs uninstrumented; a second pass of the same K steps
    # with the library's per-launch events (they cost a few per cent) gives the
    # per-kernel times behind the roofline.
    def timed_pass(first_step, profiled):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        mpc.profile_reset()
        mpc.profile_enable(profiled)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            if profiled:
                step(first_step + i, x_dev)
            else:
                graphs[i][0].replay()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        mpc.profile_enable(False)
        return [a.elapsed_time(b) for a, b in ev]

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    step_ms = timed_pass(0, False)
    clk = clocks.stop()
    prof_step_ms = timed_pass(args.steps, True)
    prof = {k: mpc.profile_read(k) for k in ("gemm_plain", "gemm_limb", "limb_planes",
                                                 "private_relu", "private_relu_fused")}
    busy = {k: mpc.profile_busy(k) for k in prof}
    total_ms = float(sum(step_ms))
    t_max = job_time(total_ms, world, dev)
    value = whole_job_rate(args.steps, world, t_max / 1e3)

    # ---- end to end through the public API with pinned host buffers ------
    # Every step uploads its input from pinned host memory and reads its
    # revealed output back.  The copies run on a copy stream, pipelined as a
    # serving loop would: the input of step i + 1 goes up (into the other of two
    # device input buffers) while step i computes, and step i's output comes
    # down while step i + 1 computes; the timed region ends when the last output
    # has landed on the host.
    x_host = torch.from_numpy(x).pin_memory()
    out_host = torch.empty(tuple(net.out_real.shape), dtype=torch.float64).pin_memory()
    x_bufs = [torch.empty_like(x_dev), torch.empty_like(x_dev)]
    e2e_steps = max(3, args.steps)
    e2e_scheds = [synth.speech_schedule(len(ws), step=3000 + i) for i in range(e2e_steps + 3)]
    e2e_all = net.capture_pipelined(x_bufs, e2e_scheds[:-1], e2e_scheds[1:])
    net.deal(e2e_scheds[0], 0, join=True)
    for w in range(2):           # untimed: upload and warm the first two steps
        x_bufs[w].copy_(x_host, non_blocking=True)
        e2e_all[w][0].replay()
    e2e_graphs = e2e_all[2:]     # graph i (of these) reads x_bufs[i % 2]
    copy_stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_stop = torch.cuda.Event(enable_timing=True)
    up = [torch.cuda.Event() for _ in range(e2e_steps)]
    done = [torch.cuda.Event() for _ in range(e2e_steps)]
    e_start.record(stream)
    copy_stream.wait_stream(stream)
    with torch.cuda.stream(copy_stream):
        x_bufs[0].copy_(x_host, non_blocking=True)  # step 0's input
        up[0].record(copy_stream)
    for i in range(e2e_steps):
        g, out = e2e_graphs[i]
        stream.wait_event(up[i])
        g.replay()
        done[i].record(stream)
        with torch.cuda.stream(copy_stream):
            if i + 1 < e2e_steps:
                # step i + 1's input goes to the buffer step i - 1 read
                if i >= 1:
                    copy_stream.wait_event(done[i - 1])
                x_bufs[(i + 1) % 2].copy_(x_host, non_blocking=True)
                up[i + 1].record(copy_stream)
            copy_stream.wait_event(done[i])
            out_host.copy_(out, non_blocking=True)    # step i's revealed output
    stream.wait_stream(copy_stream)
    e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_s = job_time(max(time.perf_counter() - t0, e_start.elapsed_time(e_stop) / 1e3), world,
                     dev)
    e2e = {"value": whole_job_rate(e2e_steps, world, e2e_s), "unit": "samples/s",
           "h2d_bytes_per_step": int(x_host.numel() * 8),
           "d2h_bytes_per_step": int(out_host.numel() * 8)}

    # ---- the two phases alone: the online phase on triples dealt beforehand,
    # and one forward's dealing, each as a CUDA-graph replay (L2 flushed) ---
    phases = None
    if world == 1:
        sch = synth.speech_schedule(len(ws), step=5000)
        net.deal(sch, 0, join=True)

        def phase_graph(fn):
            cs = torch.cuda.Stream(device=dev)
            cs.wait_stream(stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(cs):
                with torch.cuda.graph(g, stream=cs):
                    fn()
            stream.wait_stream(cs)
            return g

        g_on = phase_graph(lambda: net.reveal(net.online(x_dev, sch, 0, wait_dealer=False)))
        g_deal = phase_graph(lambda: net.deal(sch, 1, join=True))
        phases = {"online_only_ms": median_event_ms(g_on.replay, args.steps, flush, warm=2),
                  "dealer_only_ms": median_event_ms(g_deal.replay, args.steps, flush, warm=2),
                  "pipelined_step_ms": float(np.median(step_ms)),
                  "note": "online phase of one forward on triples dealt (and convolutions "
                          "prepared) beforehand, and one forward's dealing with the "
                          "preparation, each alone as a graph replay; the timed steps "
                          "overlap the two on two streams"}
        del g_on, g_deal
        # Per-kernel busy time of the online phase alone (eager, instrumented):
        # what of the step's kernel time sits on the online critical path.
        mpc.profile_reset()
        mpc.profile_enable(True)
        for _ in range(3):
            flush.zero_()
            net.reveal(net.online(x_dev, sch, 0, wait_dealer=False))
        torch.cuda.synchronize()
        mpc.profile_enable(False)
        phases["online_kernel_busy_ms"] = {
            k: mpc.profile_busy(k) / 3 for k in ("gemm_limb", "limb_planes", "private_relu_fused")
            if mpc.profile_read(k)[0]}
        # The same with the convolutions' input-independent half left in the
        # online phase (no prepared planes): the split the timed steps do not use.
        was_prepared = net.prepared
        net.enable_prepared(not was_prepared)
        if net.prepared != was_prepared:
            key = "prepared" if net.prepared else "unprepared"
            net.deal(sch, 0, join=True)
            g_on = phase_graph(lambda: net.reveal(net.online(x_dev, sch, 0, wait_dealer=False)))
            g_deal = phase_graph(lambda: net.deal(sch, 1, join=True))
            phases[f"online_only_{key}_ms"] = median_event_ms(g_on.replay, args.steps, flush,
                                                              warm=2)
            phases[f"dealer_only_{key}_ms"] = median_event_ms(g_deal.replay, args.steps, flush,
                                                              warm=2)
            del g_on, g_deal
        net.enable_prepared(was_prepared)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    # The limb GEMM launches run 40-90 us each inside a ~1.4 ms step and a timed
    # region of tens of ms, far from the seconds-long loop behind the sustained
    # figure: the burst peak is their denominator.
    bf16_peak = peaks.get("bf16_tflops", 1800.0)
    peak_src = "of measured" if peaks else "of fallback"

    macs = layer_macs(net)
    n_relu = sum(b["n"] for b in net.bufs)
    # dominant kernel by summed device time
    kern = max(prof, key=lambda k: prof[k][1])
    launches, kms_sum = prof[kern]
    # achieved = algorithmic work of all launches / the time they were running.
    # Launches on the dealer stream overlap the main stream's, so the summed
    # per-launch durations count shared time twice; the union of the launch
    # intervals (busy time) counts it once.  Both are reported.
    kms = busy[kern]
    if kern in ("private_relu", "private_relu_fused"):
        # the fused kernel moves only x and y; its algorithmic bytes are still
        # reported against the unfused protocol's 672 B/element
        achieved = relu_bytes_per_elem() * n_relu * args.steps / (kms / 1e3) / 1e9
        roof = {"kernel": kern, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                "peak_source": peak_src + " (copy bandwidth)"}
    elif kern == "gemm_limb":
        achieved = 36 * 2 * macs * args.steps / (kms / 1e3) / 1e12   # limb-pair MMA flops
        roof = {"kernel": kern, "bound": "tensor", "achieved": achieved, "peak": bf16_peak,
                "unit": "TFLOP/s", "frac": achieved / bf16_peak,
                "traffic": LIMB_GEMM_DRAM_BYTES_PER_LAUNCH,
                "traffic_note": "bytes per launch, mean of the 8 limb GEMM launches of one "
                                "step (dram__bytes_read.sum + dram__bytes_write.sum, ncu); "
                                "the digit planes they read are "
                                f"{LIMB_GEMM_PLANE_BYTES_PER_LAUNCH / 1e6:.1f} MB per launch",
                "ncu_tensor_active_pct": LIMB_GEMM_TENSOR_ACTIVE_SPEECH,
                "ncu_tensor_active_note": "sm__pipe_tensor_cycles_active of an online "
                                          "speech-layer launch, one ncu capture (serialised)",
                "ncu_tensor_active_step_pct": LIMB_GEMM_TENSOR_ACTIVE_SPEECH_STEP,
                "peak_source": peak_src + " (bf16 burst)",
                "launches_per_step": launches / args.steps,
                "busy_ms_per_step": kms / args.steps,
                "launch_ms_sum_per_step": kms_sum / args.steps}
    else:
        # Plain engine: bound by 32-bit integer multiply-add issue.  Peak ring MAC
        # rate = 148 SMs x 64 IMAD/clk x 2.032 GHz / 4 IMAD slots per ring MAC.
        peak_tops = 148 * 64 * 2.032e9 / 4 * 2 / 1e12
        achieved = 2 * macs * args.steps / (kms / 1e3) / 1e12
        roof = {"kernel": kern, "bound": "alu", "achieved": achieved, "peak": peak_tops,
                "unit": "TOPS", "frac": achieved / peak_tops, "traffic": None,
                "peak_source": "derived: 148 SM x 64 IMAD/clk x 2.032 GHz / 4 IMAD per ring MAC"}

    extras = {}
    if not args.no_extras and world == 1:
        # Further measurements on the same box, after the timed region: the
        # limb-vs-plain ring GEMM, the HBM-bound kernels, the ResNet-18 and
        # batched workloads (each bounded to a few seconds).
        extras["gemm_sweep"] = extra_gemm_sweep(dev, peaks)
        extras["hbm_kernels"] = extra_hbm_kernels(dev, peaks, [1 << 26])
        extras["resnet18"] = extra_resnet(dev, peaks, steps=3, warmup=1)
        extras["batched"] = extra_batched(dev, reps=5)

    cpu = None
    if not args.no_cpu_baseline and world == 1:   # host baseline: rank 0 at N = 1 only
        cpu = cpu_baseline_measure()
        if not args.no_extras:
            # the oracle on bounded samples of the ring GEMM and ResNet workloads
            cpu["other_workloads"] = {"ring_gemm": oracle_gemm_measure(),
                                      "resnet18": oracle_resnet_measure()}

    gemm_ms = busy["gemm_plain"] + busy["gemm_limb"]
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "parties": 2, "batch": 1, "engine": args.algo,
                   "dealer": "one step ahead on a low-priority stream, every step dealing one "
                             "forward: the seven layers' convolution triples in one batched "
                             "call (one limb GEMM launch), then each convolution's "
                             "input-independent half prepared (F = W - B opened, weight-side "
                             "and im2col(A_p) digit planes)",
                   "l2": "flushed between steps (256 MiB write outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "ring_gemm_tops": 2 * macs * args.steps / (gemm_ms / 1e3) / 1e12 if gemm_ms else None,
        "ring_macs_per_step": macs,
        "relu_elements_per_step": n_relu,
        "step_ms": {"min": min(step_ms), "median": float(np.median(step_ms)),
                    "max": max(step_ms)},
        "profiled_pass_ms_per_step": float(sum(prof_step_ms)) / args.steps,
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items() if v[0]},
        "kernel_busy_ms_per_step": {k: busy[k] / args.steps for k, v in prof.items() if v[0]},
        "clocks": clk,
        "phases": phases,
        "e2e": e2e,
        "gpu_launches": int(stats["launches"]),
        "roofline": roof,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- extras
# ALU roof of the plain engine: 148 SMs x 64 32-bit IMAD/clk x 2.032 GHz, 4 IMAD
# issue slots per 64-bit ring MAC (lo x lo wide = 2, two cross products = 2).
PLAIN_PEAK_TOPS = 148 * 64 * 2.032e9 / 4 * 2 / 1e12
# Algorithmic HBM bytes per element of the two-party kernels (triples materialised):
#   beaver_mul + trunc: read X, Y, A, B, C (5 x 16 B), write Z (16 B) = 96
#   truncate (in place): read + write 16 B = 32
#   a2b: read 16 B, 12 AND gates x (a, b, c) x 2 words = 576 B, write 16 B = 608
#   private_relu: relu_bytes_per_elem() = 672.25


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def median_event_ms(fn, reps, flush=None, warm=1):
    """Median device time (ms) of fn over `reps` calls, CUDA events on the current
    stream, with `warm` untimed calls first and the L2 flushed before each timed
    call when a flush buffer is given."""
    import torch
    stream = torch.cuda.current_stream()
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        ts.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ts]))


def measure_ring_gemm(n, algo, dev, reps, flush, bf16_burst):
    """One ring GEMM Z = A B, M = N = K = n, words uniform over Z/2^64 (seeded)."""
    import torch

    import paper_2109_00984_b300 as mpc
    g = torch.Generator(device=dev)
    g.manual_seed(n)
    A = torch.randint(-2 ** 63, 2 ** 63 - 1, (n, n), dtype=torch.int64, device=dev, generator=g)
    B = torch.randint(-2 ** 63, 2 ** 63 - 1, (n, n), dtype=torch.int64, device=dev, generator=g)
    Z = torch.empty((n, n), dtype=torch.int64, device=dev)
    ws = torch.empty(max(1, mpc.ring_gemm_workspace_size(n, n, n, algo)), dtype=torch.uint8,
                     device=dev)

    def call():
        mpc.ring_gemm(A, B, None, algo=algo, out=Z, ws=ws)

    ms = median_event_ms(call, reps, flush)
    rec = {"ms": ms, "ring_tops": 2 * n ** 3 / (ms / 1e3) / 1e12, "reps": reps}
    if algo == mpc.LIMB:
        mpc.profile_reset()
        mpc.profile_enable(True)
        for _ in range(reps):
            flush.zero_()
            call()
        torch.cuda.synchronize()
        mpc.profile_enable(False)
        kl, kms = mpc.profile_read("gemm_limb")
        pl, pms = mpc.profile_read("limb_planes")
        k_ms = kms / max(kl, 1)
        rec["mma_kernel_ms"] = k_ms
        rec["planes_ms"] = pms / max(pl, 1)
        rec["tensor_tflops"] = 72 * n ** 3 / (k_ms / 1e3) / 1e12   # 36 digit-pair MMAs per MAC
        rec["tensor_frac"] = rec["tensor_tflops"] / bf16_burst
        rec["tensor_frac_peak"] = "bf16 burst (the kernel is timed alone)"
        if n == 4096:
            rec["ncu_tensor_active_pct"] = LIMB_GEMM_TENSOR_ACTIVE_4096
    else:
        rec["alu_frac"] = rec["ring_tops"] / PLAIN_PEAK_TOPS
        rec["alu_peak_ring_tops"] = PLAIN_PEAK_TOPS
    del A, B, Z, ws
    torch.cuda.empty_cache()
    return rec


def measure_beaver3(n, algo, dev, reps, flush):
    """The three-party Beaver online step on an n x n x n product (the GEMM sweep's 3-party case):
    opening of E and F, then per party one ring GEMM over the K-concatenated pairs
    [E | A_p] [B_p (+ F) ; F] (K' = 2n), plus C_p and the truncation; triples dealt
    beforehand.  Ring ops = 2 x 3 parties x n^2 x 2n."""
    import torch

    import paper_2109_00984_b300 as mpc
    P = 3
    g = torch.Generator(device=dev)
    g.manual_seed(n + 3)
    X = torch.randint(-2 ** 63, 2 ** 63 - 1, (P, n, n), dtype=torch.int64, device=dev, generator=g)
    Y = torch.randint(-2 ** 63, 2 ** 63 - 1, (P, n, n), dtype=torch.int64, device=dev, generator=g)
    A, B, C = mpc.ttp_matmul_triple(P, n, n, n, 1, 70000 + n, algo=mpc.LIMB, device=dev)
    Z = torch.empty((P, n, n), dtype=torch.int64, device=dev)
    ws = torch.empty(max(1, mpc.matmul_workspace_size(P, n, n, n, algo)), dtype=torch.uint8,
                     device=dev)

    def call():
        mpc.beaver_matmul(X, Y, A, B, C, algo=algo, trunc_bits=16, out=Z, ws=ws)

    ms = median_event_ms(call, reps, flush)
    ring_ops = 2.0 * P * n * n * 2 * n
    rec = {"ms": ms, "ring_tops": ring_ops / (ms / 1e3) / 1e12, "reps": reps}
    del X, Y, A, B, C, Z, ws
    torch.cuda.empty_cache()
    return rec


def extra_gemm_sweep(dev, peaks, sizes=(4096, 8192), reps=5):
    """Limb (tcgen05) vs plain (CUDA-core) ring GEMM at the largest sweep sizes."""
    import torch

    import paper_2109_00984_b300 as mpc
    burst = peaks.get("bf16_tflops", 1800.0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    out = {"workload": "ring GEMM M=N=K, uniform Z/2^64 words, L2 flushed between launches; "
                       "limb: whole call (digit planes + MMA kernel); tensor_frac: MMA kernel "
                       "at 72 n^3 digit-pair flops against the measured bf16 burst peak; "
                       "plain: against its derived ALU roof "
                       f"({PLAIN_PEAK_TOPS:.2f} ring TOPS)"}
    for n in sizes:
        limb = measure_ring_gemm(n, mpc.LIMB, dev, reps, flush, burst)
        plain = measure_ring_gemm(n, mpc.PLAIN, dev, max(2, reps // 2), flush, burst)
        out[str(n)] = {"limb": limb, "plain": plain, "limb_over_plain": plain["ms"] / limb["ms"]}
    # The three-party Beaver online step at the first size, both engines.
    n = sizes[0]
    b_limb = measure_beaver3(n, mpc.LIMB, dev, reps, flush)
    b_plain = measure_beaver3(n, mpc.PLAIN, dev, 2, flush)
    out[f"beaver3_{n}"] = {"workload": "three-party Beaver matmul online step (E, F opened, "
                                       "per party one two-pair ring GEMM, K' = 2n, C and "
                                       "truncation), triples dealt beforehand",
                           "limb": b_limb, "plain": b_plain,
                           "limb_over_plain": b_plain["ms"] / b_limb["ms"]}
    del flush
    torch.cuda.empty_cache()
    return out


def measure_hbm_kernels(dev, peaks, n, reps=5):
    """The HBM-bound two-party kernels on n elements (inputs far larger than L2 from
    n = 2^24 on, so no flush), GB/s of algorithmic bytes against the copy peak."""
    import torch

    import paper_2109_00984_b300 as mpc
    hbm = peaks.get("hbm_gbs", 6400.0)
    g = torch.Generator(device=dev)
    g.manual_seed(5)

    def words(shape):
        return torch.randint(-2 ** 63, 2 ** 63 - 1, shape, dtype=torch.int64, device=dev,
                             generator=g)

    def rec(name, ms, bpe):
        gbs = bpe * n / (ms / 1e3) / 1e9
        return {"ms": ms, "bytes_per_elem": bpe, "gbs": gbs, "frac": gbs / hbm}

    res = {}
    X, Y = words((2, n)), words((2, n))
    A, B, C = mpc.ttp_mul_triple(2, n, 1, 11, device=dev)
    Z = torch.empty_like(X)
    res["beaver_mul_trunc"] = rec("beaver_mul_trunc", median_event_ms(
        lambda: mpc.beaver_mul(X, Y, A, B, C, trunc_bits=16, out=Z), reps), 96.0)
    res["truncate"] = rec("truncate", median_event_ms(lambda: mpc.truncate(Z, 16), reps), 32.0)
    del Y, A, B, C
    T = mpc.ttp_and_triples(2, n, 1, 12, device=dev)
    res["a2b"] = rec("a2b", median_event_ms(lambda: mpc.a2b(X, T, 1, 13, out=Z), reps), 608.0)
    ra, rb = mpc.ttp_b2a_bits(2, n, 1, 14, device=dev)
    MT = torch.empty((3, 2, n), dtype=torch.int64, device=dev)
    mpc.ttp_mul_triple(2, n, 1, 15, out=(MT[0], MT[1], MT[2]))
    res["private_relu"] = rec("private_relu", median_event_ms(
        lambda: mpc.private_relu(X, T, ra, rb, MT, 1, 16, out=Z), reps), relu_bytes_per_elem())
    del X, Z, T, ra, rb, MT
    torch.cuda.empty_cache()
    return res


def extra_hbm_kernels(dev, peaks, sizes, reps=5):
    out = {"workload": "two-party HBM-bound kernels, triples materialised; GB/s of algorithmic "
                       "bytes per element (beaver_mul+trunc 96, truncate 32, a2b 608, "
                       f"private_relu {relu_bytes_per_elem():.2f}) against the measured copy "
                       "bandwidth; inputs > L2"}
    for n in sizes:
        out[f"2^{int(np.log2(n))}"] = measure_hbm_kernels(dev, peaks, n, reps)
    return out


def run_gemm_sweep(args):
    """Ring GEMM Z = A B over Z/2^64, M = N = K = n, words uniform over the ring.

    Times each engine with CUDA events (L2 flushed between launches) and reports
    ring TOPS = 2 n^3 / t; for the limb engine also the tensor-pipe rate
    72 n^3 / t (36 bf16 digit-pair products per ring MAC) against the bf16 peak.
    """
    import torch

    import paper_2109_00984_b300 as mpc

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    bf16 = peaks.get("bf16_tflops", 1800.0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    algos = {"plain": [mpc.PLAIN], "limb": [mpc.LIMB], "auto": [mpc.PLAIN, mpc.LIMB]}[args.algo]
    out = {}
    for n in [int(v) for v in args.sizes.split(",")]:
        rng = np.random.default_rng(0)
        A = torch.from_numpy(rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64).view(np.int64)).to(dev)
        B = torch.from_numpy(rng.integers(0, 2 ** 64, (n, n), dtype=np.uint64).view(np.int64)).to(dev)
        Z = torch.empty((n, n), dtype=torch.int64, device=dev)
        for algo in algos:
            name = "limb" if algo == mpc.LIMB else "plain"
            ws = torch.empty(max(1, mpc.ring_gemm_workspace_size(n, n, n, algo)), dtype=torch.uint8,
                             device=dev)
            reps = max(1, min(args.steps, int(2e12 // (n ** 3)) + 1))
            mpc.ring_gemm(A, B, None, algo=algo, out=Z, ws=ws)
            torch.cuda.synchronize()
            mpc.profile_reset()
            mpc.profile_enable(True)
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                mpc.ring_gemm(A, B, None, algo=algo, out=Z, ws=ws)
                e1.record()
                ts.append((e0, e1))
            torch.cuda.synchronize()
            mpc.profile_enable(False)
            ms = float(np.median([a.elapsed_time(b) for a, b in ts]))
            rec = {"ms": ms, "ring_tops": 2 * n ** 3 / (ms / 1e3) / 1e12, "reps": reps}
            if algo == mpc.LIMB:
                kl, kms = mpc.profile_read("gemm_limb")
                pl, pms = mpc.profile_read("limb_planes")
                rec["mma_kernel_ms"] = kms / max(kl, 1)
                rec["planes_ms"] = pms / max(pl, 1)
                tf = 72 * n ** 3 / (rec["mma_kernel_ms"] / 1e3) / 1e12
                rec["tensor_tflops"] = tf
                rec["tensor_frac_of_bf16_burst"] = tf / bf16
            out[f"{name}_{n}"] = rec
            out[f"beaver3_{name}_{n}"] = measure_beaver3(n, algo, dev, min(reps, 3), flush)
            del ws
        del A, B, Z
        torch.cuda.empty_cache()
    print(json.dumps({"workload": "ring GEMM sweep M=N=K, uniform Z/2^64 words",
                      "bf16_peak_tflops": bf16, "results": out}), flush=True)


def run_batched(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps(measure_batched(dev, max(3, min(args.steps, 10)), args.batch_count)),
          flush=True)


def extra_batched(dev, reps=3):
    r = measure_batched(dev, reps)
    return r


def measure_batched(dev, reps, count=512):
    """512 two-party Beaver matmuls with (M, N, K) log-uniform in [32, 2048] (seed 2).

    Times the online step (opening + products + truncation; triples dealt
    beforehand) three ways with CUDA events, L2 flushed between repetitions:
    one beaver_matmul call per product, one batched call, and the batched call
    captured once in a CUDA graph and replayed.
    """
    import torch

    import paper_2109_00984_b300 as mpc

    P = 2
    dims = synth.batched_dims()[:count]
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    prods = []
    for i, (M, N, K) in enumerate(dims):
        M, N, K = int(M), int(N), int(K)
        X = torch.randint(-2 ** 63, 2 ** 63 - 1, (P, M, K), dtype=torch.int64, device=dev, generator=gen)
        Y = torch.randint(-2 ** 63, 2 ** 63 - 1, (P, K, N), dtype=torch.int64, device=dev, generator=gen)
        A, B, C = mpc.ttp_matmul_triple(P, M, N, K, 1, 10000 + i, algo=mpc.AUTO, device=dev)
        Z = torch.empty((P, M, N), dtype=torch.int64, device=dev)
        prods.append((X, Y, A, B, C, Z))
    ring_ops = float(sum(2 * P * 2 * int(M) * int(N) * int(K) for M, N, K in dims))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in ts]))

    # (a) one call per product (the engine AUTO picks per shape)
    ws = {}

    def per_product():
        for (X, Y, A, B, C, Z) in prods:
            key = (X.shape, Y.shape)
            w = ws.get(key)
            if w is None:
                M, K = X.shape[1], X.shape[2]
                w = ws[key] = torch.empty(max(1, mpc.matmul_workspace_size(P, M, Y.shape[2], K, mpc.AUTO)),
                                          dtype=torch.uint8, device=dev)
            mpc.beaver_matmul(X, Y, A, B, C, algo=mpc.AUTO, trunc_bits=16, out=Z, ws=w)

    per_product()
    t_each = timed(per_product, reps)

    # (b) one batched call, autotuned routing
    bm = mpc.BatchedMatmul(prods, algo=mpc.AUTO, trunc_bits=16)
    tune = bm.autotune()
    bm.ensure_workspace(dev)
    bm()
    mpc.reset_stats()
    t_batched = timed(bm, reps)
    launches = mpc.get_stats()["launches"] / reps

    # per-kernel device time of one batched call (the library's launch events)
    mpc.profile_reset()
    mpc.profile_enable(True)
    for _ in range(reps):
        flush.zero_()
        bm()
    torch.cuda.synchronize()
    mpc.profile_enable(False)
    kernels = {}
    for k in ("batched_open", "gemm_plain_batched", "limb_planes", "gemm_limb"):
        n_l, ms_k = mpc.profile_read(k)
        if n_l:
            kernels[k] = ms_k / reps
    limb_macs = float(sum(2 * P * int(M) * int(N) * int(K) for M, N, K in dims
                          if float(M) * float(N) * float(K) >= tune.limb_min_macs))

    # (c) the batched call captured in a CUDA graph
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            bm()
    torch.cuda.synchronize()
    g.replay()
    t_graph = timed(g.replay, reps)

    line = {"workload": f"{count} uneven 2-party Beaver matmuls, (M,N,K) log-uniform in "
                        "[32,2048] (seed 2), truncation 2^16, online step (triples dealt "
                        "beforehand)",
            "ring_ops_per_batch": ring_ops,
            "per_product_ms": t_each, "batched_ms": t_batched, "graph_ms": t_graph,
            "per_product_ring_tops": ring_ops / (t_each / 1e3) / 1e12,
            "batched_ring_tops": ring_ops / (t_batched / 1e3) / 1e12,
            "graph_ring_tops": ring_ops / (t_graph / 1e3) / 1e12,
            "speedup_graph_vs_per_product": t_each / t_graph,
            "tuned_limb_min_macs": tune.limb_min_macs,
            "kernel_ms_per_call": kernels,
            "limb_tensor_frac": (72 * limb_macs / (kernels["gemm_limb"] / 1e3) / 1e12 /
                                 load_peaks().get("bf16_tflops", 1800.0))
            if kernels.get("gemm_limb") else None,
            "kernel_launches_per_batched_call": launches}
    del prods, bm, g
    torch.cuda.empty_cache()
    return line


def run_resnet(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    print(json.dumps(measure_resnet(dev, load_peaks(), args.steps, args.warmup)), flush=True)


def extra_resnet(dev, peaks, steps=3, warmup=1):
    r = measure_resnet(dev, peaks, steps, warmup)
    r.pop("clocks", None)
    return r


def measure_resnet(dev, peaks, steps_arg, warmup):
    """Private inference of the ResNet-18-shaped CNN: 2 parties, batch 8 of 3x224x224.

    One step = share the batch, deal and consume all material of every layer
    (convolutions, ReLUs, max-pool tree, residual adds, average pool, FC),
    reveal the logits.  Device-timed with CUDA events, L2 flushed between steps.
    """
    import torch

    import paper_2109_00984_b300 as mpc
    from paper_2109_00984_b300.resnet import PrivateResNet18

    batch = 8
    x = torch.from_numpy(synth.resnet_input(batch=batch, hw=224)).to(dev)
    sched = synth.resnet_schedule()
    net = PrivateResNet18(synth.resnet_weights(), synth.RESNET18, sched, algo=mpc.AUTO, device=dev,
                          prepare_weights=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for w in range(max(1, warmup)):
        net.reveal(net.forward(x, synth.resnet_schedule(step=100 + w)))
    torch.cuda.synchronize()
    steps = max(1, steps_arg)

    def timed_pass(first_step, profiled):
        mpc.profile_reset()
        mpc.profile_enable(profiled)
        mpc.reset_stats()
        ts = []
        for i in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if profiled:
                net.reveal(net.forward(x, synth.resnet_schedule(step=first_step + i)))
            else:
                graphs[i][0].replay()
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        mpc.profile_enable(False)
        return float(sum(a.elapsed_time(b) for a, b in ts)) / steps

    # Headline: replays of one CUDA graph per step (each with its own schedule);
    # the launch count is taken while they are captured.
    mpc.reset_stats()
    graphs = net.capture(x, [synth.resnet_schedule(step=i) for i in range(steps)])
    stats = mpc.get_stats()
    graphs[0][0].replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.5)
    ms = timed_pass(0, False)     # headline: uninstrumented graph replays
    clk = clocks.stop()
    timed_pass(steps, True)       # per-kernel times
    prof = {k: mpc.profile_read(k) for k in ("gemm_plain", "gemm_limb", "limb_planes",
                                                 "private_relu", "private_relu_fused",
                                                 "gemm_plain_batched")}
    busy = {k: mpc.profile_busy(k) for k in prof}
    # Every ResNet-18 product at batch 8 is above the AUTO threshold, so all ring
    # MACs run on the limb engine: the online products count P x 2 pairs x MNK
    # (the library counter), the dealer's c = a b one pair more per product.
    online_macs = stats["ring_macs"] / steps
    limb_macs = online_macs * (1 + 1 / 4)
    kern = max(busy, key=lambda k: busy[k])
    roof = {"kernel": kern, "busy_ms_per_step": busy[kern] / steps}
    relu_elems = stats["and_gates"] / 12 / steps      # 12 secret ANDs per two-party ReLU
    if kern == "gemm_limb":
        tf = 72 * limb_macs / (busy[kern] / steps / 1e3) / 1e12
        roof.update({"bound": "tensor", "achieved": tf, "unit": "TFLOP/s",
                     "peak": peaks.get("bf16_tflops", 1800.0),
                     "frac": tf / peaks.get("bf16_tflops", 1800.0),
                     "peak_source": "of measured (bf16 burst)"})
    elif kern == "private_relu_fused":
        # ALU-bound: 17 Philox4x64-10 blocks regenerated per element
        gb = RELU_FUSED_BLOCKS * relu_elems / (busy[kern] / steps / 1e3) / 1e9
        roof.update({"bound": "alu", "achieved": gb, "unit": "G Philox blocks/s",
                     "peak": PHILOX_PEAK_BLOCKS / 1e9, "frac": gb * 1e9 / PHILOX_PEAK_BLOCKS,
                     "peak_source": "derived: 64 32-bit multiply results/clk/SM, 148 SMs, "
                                    "2032 MHz, 160 per Philox4x64-10 block"})
    if "gemm_limb" in busy and kern != "gemm_limb":
        tf = 72 * limb_macs / (busy["gemm_limb"] / steps / 1e3) / 1e12
        roof["gemm_limb_tensor_frac"] = tf / peaks.get("bf16_tflops", 1800.0)
    line = {"workload": "private ResNet-18-shaped inference, 2 parties, batch 8 x 3x224x224, "
                        "He-init weights, dealer (with the convolutions' preparation) in the "
                        "step, one CUDA-graph replay per step",
            "value": batch / (ms / 1e3), "unit": "images/s", "ms_per_step": ms, "steps": steps,
            "paper_context_images_per_s": 1 / 2.49,
            "kernel_ms_per_step": {k: v[1] / steps for k, v in prof.items() if v[0]},
            "kernel_busy_ms_per_step": {k: busy[k] / steps for k, v in prof.items() if v[0]},
            "ring_macs_per_step": online_macs + online_macs / 4,
            "relu_elements_per_step": relu_elems,
            "roofline": roof,
            "gpu_launches_per_step": stats["launches"] / steps, "clocks": clk}
    del net, graphs
    torch.cuda.empty_cache()
    return line


# Philox4x64-10 blocks the fused private ReLU regenerates per element (one
# quad_gen = one block per element): the A2B masks 1, the AND gates' a/b words
# 12, their c_0 words 3, the B2A pair (with the triple's c_0) 1, the triple's
# a/b words 1.
RELU_FUSED_BLOCKS = 18
# Philox4x64-10 blocks each fused function regenerates per element (one quad_gen
# call = one block per element): exp = 2 chunks of 3; a product = 5/4, a square
# = 3/4; a comparison = 16; see the kernels' word lists.
APPROX_BLOCKS = {"exp": 6, "reciprocal": 50, "sigmoid": 50, "tanh": 50, "erf": 12,
                 "inv_sqrt": 49, "log": 54}
# ALU roofline of a fused-dealer kernel: a Philox4x64-10 block is 10 rounds of two
# 64x64->128-bit products, each 4 wide 32x32->64 partial products = 8 32-bit
# multiply results, i.e. 160 per block; 64 such results per clock per SM.
PHILOX_PEAK_BLOCKS = 64 * 148 * 2032e6 / 160


def run_approx(args):
    """Fused function approximations (two parties) on 2^25 elements each, and the
    ViT-B/16 attention softmax (12 layers x 12 heads x 197 rows of 197 per image).

    Inputs (1 GiB of shares per function) exceed L2, so no flush is needed.
    """
    import torch

    import paper_2109_00984_b300 as mpc

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = 1 << 25
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    domains = {"exp": (-6, 3), "reciprocal": (-30, 30), "sigmoid": (-12, 12), "tanh": (-5, 5),
               "erf": (-1.5, 1.5), "inv_sqrt": (0.01, 100), "log": (0.01, 100)}
    calls = {"exp": mpc.exp, "reciprocal": mpc.reciprocal, "sigmoid": mpc.sigmoid,
             "tanh": mpc.tanh, "erf": mpc.erf, "inv_sqrt": mpc.inv_sqrt, "log": mpc.log}
    stream = torch.cuda.current_stream()
    steps = max(1, args.steps)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    clocks = ClockSampler(0)
    clocks.start()
    funcs = {}
    for name, (lo, hi) in domains.items():
        x = torch.rand(n, generator=g, device=dev, dtype=torch.float64) * (hi - lo) + lo
        X = mpc.ring_share(x, 2, 0, 7, 1)
        Y = torch.empty_like(X)
        ms = timed(lambda: calls[name](X, 7, 100, out=Y))
        rate = n / (ms / 1e3)
        funcs[name] = {"ms": ms, "elements_per_s": rate,
                       "philox_blocks_per_s": rate * APPROX_BLOCKS[name],
                       "alu_frac": rate * APPROX_BLOCKS[name] / PHILOX_PEAK_BLOCKS}
        del X, Y, x
    # ViT-B/16 attention softmax, one image: 144 heads x 197 rows of 197 logits
    rows, m = 12 * 12 * 197, 197
    logits = torch.randn(rows, m, generator=g, device=dev, dtype=torch.float64) * 2
    S = mpc.ring_share(logits, 2, 0, 7, 2)
    Ys = torch.empty_like(S)
    ws = torch.empty(mpc._lib.load().mpc_softmax_workspace_size(2, rows, m), dtype=torch.uint8,
                     device=dev)
    mpc.reset_stats()
    sm_ms = timed(lambda: mpc.softmax(S, 7, 100, out=Ys, ws=ws))
    stats = mpc.get_stats()
    clk = clocks.stop()
    # blocks per logit: the max tree's ReLUs (17 per pair, m - 1 pairs per row), exp (6),
    # the final product (2), the reciprocal per row (31)
    sm_blocks = rows * (17 * (m - 1) + 6 * m + 2 * m + 31)
    head = funcs["sigmoid"]
    line = {"metric": "fused private sigmoid throughput (2 parties, Z/2^64, 2^16 fixed point)",
            "value": head["elements_per_s"], "unit": "elements/s", "higher_is_better": True,
            "steps": steps, "warmup": max(3, args.warmup), "dtype": "u64",
            "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "function approximations, 2^25 elements each, inputs > L2 "
                                   "(no flush); ViT-B/16 softmax 28368 rows x 197",
                       "exp_iters": 8, "nr_iters": 10, "erf_terms": 8, "log_iters": 3,
                       "log_order": 8},
            "roofline": {"bound": "alu", "achieved": head["philox_blocks_per_s"] / 1e9,
                         "peak": PHILOX_PEAK_BLOCKS / 1e9, "unit": "G Philox blocks/s",
                         "frac": head["alu_frac"], "traffic": None,
                         "peak_source": "derived: 64 32-bit multiply results/clk/SM, 148 SMs, "
                                        "2032 MHz, 160 per Philox4x64-10 block"},
            "functions": funcs,
            "vit_softmax": {"ms_per_image": sm_ms, "images_per_s": 1e3 / sm_ms,
                            "rows": rows, "m": m,
                            "philox_blocks_per_s": sm_blocks / (sm_ms / 1e3),
                            "alu_frac": sm_blocks / (sm_ms / 1e3) / PHILOX_PEAK_BLOCKS,
                            "launches_per_call": stats["launches"] / max(1, stats["calls"]) if
                            stats.get("calls") else None,
                            "rounds_per_call": stats["rounds"] / max(1, stats["calls"]) if
                            stats.get("calls") else None},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_elementwise(args):
    """The HBM-bound kernels swept over n = 2^20 .. 2^26 (two parties)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    peaks = load_peaks()
    clocks = ClockSampler(0)
    clocks.start()
    res = extra_hbm_kernels(dev, peaks, [1 << int(e) for e in args.elem_log2.split(",")],
                            reps=max(3, args.steps))
    res["clocks"] = clocks.stop()
    print(json.dumps(res), flush=True)


def main():
    args = parse()
    if args.workload == "elementwise" and args.impl != "reference":
        run_elementwise(args)
        return
    if args.workload == "resnet" and args.impl != "reference":
        run_resnet(args)
        return
    if args.workload == "batched" and args.impl != "reference":
        run_batched(args)
        return
    if args.workload == "approx" and args.impl != "reference":
        run_approx(args)
        return
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "gemm":
        run_gemm_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
