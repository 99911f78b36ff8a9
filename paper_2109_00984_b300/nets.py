"""Private 1-D conv stack (speech-shaped) as a sequence of library calls.

Each layer runs, on the device and through the C ABI only:
  dealer:  ttp_conv2d_triple, ttp_and_triples, ttp_b2a_bits, ttp_mul_triple
  online:  beaver_conv2d (+ truncation by 2^16 fused in its epilogue),
           private_relu (A2B + Kogge-Stone + B2A + Beaver mask product)
With fused_relu (the default) the four ReLU dealer calls and private_relu are
one private_relu_fused call that regenerates the same material in registers
(bit-identical results; the schedule's and/b2a/mul/relu op ids are
consecutive).
The weights are shared once by party 1 at construction; the input is shared by
party 0 in every forward, and the output is revealed at the end (§5.1, §5.2).
All buffers are allocated up front so that a forward can be captured in a
CUDA graph.

The dealer's work depends only on shapes and op ids, never on the data, so
with overlap_dealer (the default) every layer's convolution triple is dealt on
a second stream that runs ahead of the online phase; the online convolution of
layer l waits on an event recorded after layer l's triple.  Each stream has its
own workspace.  With the limb engine the dealer stream also runs the
convolution's input-independent half right after the triple
(beaver_conv2d_prepare: opening F = W - B, the weight-side digit planes and
those of im2col(A_p)); the online phase runs beaver_conv2d_relu_prepared on them
(bit-identical to beaver_conv2d_relu).
"""
import torch

from . import api


def _same_output(a, b):
    """Convolutions whose triples one batched dealer call can deal together."""
    return (a.c_out, a.batch) == (b.c_out, b.batch) and api.conv_out_hw(a) == api.conv_out_hw(b)


class PrivateConv1dStack:
    def __init__(self, weights, strides, pads, frames, batch=1, algo=api.PLAIN, frac_bits=16,
                 weight_ops=None, seed=1, device="cuda", fused_relu=True, overlap_dealer=True,
                 prepare_weights=False, batch_triples=True, prepare_products=False):
        self.P = 2
        self.fused_relu = fused_relu
        # deal the triples of consecutive layers with one output shape in one
        # batched call (one GEMM launch for all their products on the limb engine)
        self.batch_triples = batch_triples
        self.overlap_dealer = overlap_dealer
        self.algo = algo
        self.frac_bits = frac_bits
        self.seed = seed
        self.device = device
        self.descs = []
        self.W = []
        L = frames
        for l, (w, s, p) in enumerate(zip(weights, strides, pads)):
            Cout, Cin, k = w.shape
            d = api.conv_desc(batch, Cin, 1, L, Cout, 1, k, 1, s, 0, p)
            self.descs.append(d)
            wt = torch.as_tensor(w, dtype=torch.float64, device=device).contiguous()
            op = weight_ops[l] if weight_ops is not None else 900000 + l
            self.W.append(api.ring_share(wt, self.P, 1, seed, op, frac_bits))
            L = api.conv_out_hw(d)[1]
        self.out_len = L
        self.in_shape = (batch, weights[0].shape[1], frames)
        self._alloc()
        self.enable_prepared(prepare_weights or prepare_products, products=prepare_products)

    def _alloc(self):
        P, dev = self.P, self.device
        self.X0 = torch.empty((P,) + self.in_shape, dtype=torch.int64, device=dev)
        self.bufs = []
        ws_bytes = 0
        for d in self.descs:
            ho, wo = api.conv_out_hw(d)
            n = d.batch * d.c_out * ho * wo
            b = dict(
                Z=torch.empty((P, d.batch, d.c_out, ho, wo), dtype=torch.int64, device=dev),
                Y=torch.empty((P, d.batch, d.c_out, ho, wo), dtype=torch.int64, device=dev),
                n=n,
            )
            ws_bytes = max(ws_bytes, api.conv2d_workspace_size(P, d, self.algo),
                           api.conv2d_triple_workspace_size(P, d, self.algo))
            if self.fused_relu and self.algo != api.PLAIN:
                # the prepared convolution always runs on the limb engine
                ws_bytes = max(ws_bytes, api.conv2d_workspace_size(P, d, api.LIMB))
            if not self.fused_relu:
                b.update(T=torch.empty((api.KS_GATES, 3, P, n), dtype=torch.int64, device=dev),
                         ra=torch.empty((P, n), dtype=torch.int64, device=dev),
                         rb=torch.empty((P, (n + 63) // 64), dtype=torch.int64, device=dev),
                         MT=torch.empty((3, P, n), dtype=torch.int64, device=dev))
            self.bufs.append(b)
        # Two slots of convolution triples, so that the dealer can fill one while
        # the online phase consumes the other (forward_pipelined).
        self.trip = [[dict(
            A=torch.empty((P, d.batch, d.c_in, d.h, d.w), dtype=torch.int64, device=dev),
            B=torch.empty((P, d.c_out, d.c_in, d.kh, d.kw), dtype=torch.int64, device=dev),
            C=torch.empty((P, d.batch, d.c_out) + tuple(api.conv_out_hw(d)), dtype=torch.int64,
                          device=dev)) for d in self.descs] for _ in range(2)]
        self.ready = [[None] * len(self.descs) for _ in range(2)]
        # runs of consecutive layers with one output shape: (first layer, count)
        self.deal_groups = []
        for l, d in enumerate(self.descs):
            g = self.deal_groups[-1] if self.deal_groups else None
            if (self.batch_triples and g is not None and g[1] < api.MAX_TRIPLE_BATCH and
                    _same_output(self.descs[g[0]], d)):
                self.deal_groups[-1] = (g[0], g[1] + 1)
            else:
                self.deal_groups.append((l, 1))
        for first, count in self.deal_groups:
            ws_bytes = max(ws_bytes, api.conv2d_triples_workspace_size(
                P, count, self.descs[first:first + count], self.algo))
        self.prepared = False
        self.prep_products = False
        self.prep = None
        self.ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        self.dealer_ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
        # The online phase is the critical path: it runs on a high-priority stream,
        # the dealer on a low-priority one, so freed SMs go to the online kernels.
        self.dealer_stream = torch.cuda.Stream(device=dev, priority=0) if self.overlap_dealer \
            else None
        self.online_stream = torch.cuda.Stream(device=dev, priority=-5) if self.overlap_dealer \
            else None
        self.out_real = torch.empty((self.in_shape[0], self.descs[-1].c_out, self.out_len),
                                    dtype=torch.float64, device=dev)

    def enable_prepared(self, on=True, products=False):
        """With `on` (limb engine, fused ReLU) the input-independent half of each
        convolution -- opening F = W - B, the weight-side digit planes and those
        of im2col(A_p) -- is done by the dealer right after the layer's triple,
        into a prepared-plane buffer per layer and triple slot, and the online
        phase only cuts im2col(E) before its GEMM.  That shortens the online
        phase (its latency) and, with the dealer's triples batched, also raises
        the overlapped throughput (the dealer's launches fit the online phase's
        gaps).  With `products` the dealer also computes each party's product
        A_p F into C (mpc_beaver_conv2d_prepare_products), so the online GEMM
        is one operand pair per party.  Takes effect from the next deal."""
        size = api.conv2d_prep_products_size if products else api.conv2d_prep_size
        ok = on and self.fused_relu and self.algo != api.PLAIN and all(
            size(self.P, d) > 0 for d in self.descs)
        if ok and (self.prep is None or self.prep_products != products):
            self.prep = [[torch.empty(size(self.P, d), dtype=torch.uint8, device=self.device)
                          for d in self.descs] for _ in range(2)]
            if products:
                need = max(api.conv2d_prepare_products_workspace_size(self.P, d)
                           for d in self.descs)
                if self.dealer_ws.numel() < need:
                    self.dealer_ws = torch.empty(need, dtype=torch.uint8, device=self.device)
                if self.ws.numel() < need:
                    self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)
        self.prep_products = ok and products
        self.prepared = ok

    def deal(self, schedule, slot=0, join=False):
        """Enqueue the dealer's convolution triples of every layer for `schedule`
        into triple slot `slot`, on the dealer stream (recording one event per
        layer) when the dealer overlaps, else on the current stream.  With join
        the current stream then waits for the dealer (use it when dealing ahead
        of graph replays, which do not wait on these events)."""
        seed = schedule["seed"]
        main = torch.cuda.current_stream()
        ds = self.dealer_stream if self.overlap_dealer else main
        if ds is not main:
            ds.wait_stream(main)
        ws = self.dealer_ws if ds is not main else self.ws
        with torch.cuda.stream(ds):
            for first, count in self.deal_groups:
                layers = range(first, first + count)
                outs = [(self.trip[slot][l]["A"], self.trip[slot][l]["B"], self.trip[slot][l]["C"])
                        for l in layers]
                ops = [schedule["layers"][l]["conv"] for l in layers]
                if count == 1:
                    api.ttp_conv2d_triple(self.P, self.descs[first], seed, ops[0], self.algo,
                                          out=outs[0], ws=ws)
                else:
                    api.ttp_conv2d_triples(self.P, self.descs[first:first + count], seed, ops,
                                           self.algo, outs=outs, ws=ws)
                for l in layers:
                    t = self.trip[slot][l]
                    if self.prep_products:
                        api.beaver_conv2d_prepare_products(self.W[l], t["A"], t["B"], t["C"],
                                                           self.descs[l], out=self.prep[slot][l],
                                                           ws=ws)
                    elif self.prepared:
                        api.beaver_conv2d_prepare(self.W[l], t["A"], t["B"], self.descs[l],
                                                  out=self.prep[slot][l])
                    if ds is not main:
                        ev = torch.cuda.Event()
                        ev.record(ds)
                        self.ready[slot][l] = ev
        if join and ds is not main:
            main.wait_stream(ds)

    def online(self, x, schedule, slot=0, wait_dealer=True):
        """Online phase on the triples in `slot`: share the input, then per layer
        the Beaver convolution (truncation fused) and the private ReLU.  With
        wait_dealer each layer waits on the event its triple recorded."""
        main = torch.cuda.current_stream()
        if not self.overlap_dealer:
            return self._online(x, schedule, slot, main, False)
        on = self.online_stream
        on.wait_stream(main)
        with torch.cuda.stream(on):
            X = self._online(x, schedule, slot, on, wait_dealer)
        main.wait_stream(on)
        return X

    def _join_dealer(self):
        if self.overlap_dealer:
            torch.cuda.current_stream().wait_stream(self.dealer_stream)

    def forward(self, x, schedule):
        """x: float64 CUDA tensor of the input shape. Returns output shares [P, ...].

        Deals this forward's triples and runs its online phase; with
        overlap_dealer the dealer runs ahead on its own stream."""
        if not self.overlap_dealer:
            return self._online(x, schedule, 0, torch.cuda.current_stream(), False, deal=True)
        self.deal(schedule, 0)
        X = self.online(x, schedule, 0)
        self._join_dealer()
        return X

    def forward_pipelined(self, x, schedule, slot, next_schedule, wait_dealer=True):
        """One step of a software-pipelined sequence: the online phase of
        `schedule` on the triples already dealt into `slot` (by the previous
        step, or by deal() before the first), while the dealer deals
        `next_schedule` into the other slot.  Every step still deals one forward's
        triples and runs one forward's online phase."""
        self.deal(next_schedule, 1 - slot)
        X = self.online(x, schedule, slot, wait_dealer)
        self._join_dealer()
        return X

    def _online(self, x, schedule, slot, main, wait_dealer, deal=False):
        seed = schedule["seed"]
        api.ring_share(x, self.P, 0, seed, schedule["input_op"], self.frac_bits, out=self.X0)
        X = self.X0
        for l, (d, b) in enumerate(zip(self.descs, self.bufs)):
            ops = schedule["layers"][l]
            t = self.trip[slot][l]
            if deal:
                api.ttp_conv2d_triple(self.P, d, seed, ops["conv"], self.algo,
                                      out=(t["A"], t["B"], t["C"]), ws=self.ws)
                if self.prep_products:
                    api.beaver_conv2d_prepare_products(self.W[l], t["A"], t["B"], t["C"], d,
                                                       out=self.prep[slot][l], ws=self.ws)
                elif self.prepared:
                    api.beaver_conv2d_prepare(self.W[l], t["A"], t["B"], d,
                                              out=self.prep[slot][l])
            elif wait_dealer and self.ready[slot][l] is not None:
                main.wait_event(self.ready[slot][l])
            n = b["n"]
            if self.fused_relu:
                assert (ops["b2a"], ops["mul"], ops["relu"]) == (ops["and"] + 1, ops["and"] + 2,
                                                                 ops["and"] + 3)
                # convolution + truncation + ReLU: the ReLU kernel reduces the
                # GEMM's split-K partial sums itself
                if self.prep_products:
                    api.beaver_conv2d_relu_prepared_products(
                        X, t["A"], self.prep[slot][l], d, seed, ops["and"],
                        trunc_bits=self.frac_bits, out=b["Y"], ws=self.ws)
                elif self.prepared:
                    api.beaver_conv2d_relu_prepared(X, t["A"], t["C"], self.prep[slot][l], d,
                                                    seed, ops["and"], trunc_bits=self.frac_bits,
                                                    out=b["Y"], ws=self.ws)
                else:
                    api.beaver_conv2d_relu(X, self.W[l], t["A"], t["B"], t["C"], d, seed,
                                           ops["and"], self.algo, trunc_bits=self.frac_bits,
                                           out=b["Y"], ws=self.ws)
            else:
                api.beaver_conv2d(X, self.W[l], t["A"], t["B"], t["C"], d, self.algo,
                                  trunc_bits=self.frac_bits, out=b["Z"], ws=self.ws)
                api.ttp_and_triples(self.P, n, seed, ops["and"], out=b["T"])
                api.ttp_b2a_bits(self.P, n, seed, ops["b2a"], out=(b["ra"], b["rb"]))
                MT = b["MT"]
                api.ttp_mul_triple(self.P, n, seed, ops["mul"], out=(MT[0], MT[1], MT[2]))
                api.private_relu(b["Z"], b["T"], b["ra"], b["rb"], MT, seed, ops["relu"],
                                 out=b["Y"])
            X = b["Y"]
        return X

    def reveal(self, shares):
        """Decoded float64 output, shape (batch, c_out, length)."""
        _, real = api.reveal(shares, self.frac_bits, ring=False, real=True)
        return real.view(self.out_real.shape)

    def capture(self, x, schedules):
        """Capture one CUDA graph per schedule of a whole private forward + reveal.

        x is the (device) input buffer the graphs read; copy each batch into it
        before replaying.  Every graph keeps its own op ids (fresh dealer
        material per step); a replay re-runs every kernel of the step, dealer
        included, on both streams, with one host call.  Returns a list of
        (graph, revealed output) pairs.
        """
        out = []
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream(device=self.device)
        cs.wait_stream(main)
        with torch.cuda.stream(cs):
            for sched in schedules:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cs):
                    y = self.reveal(self.forward(x, sched))
                out.append((g, y))
        main.wait_stream(cs)
        return out

    def capture_pipelined(self, x, schedules, next_schedules):
        """One CUDA graph per step of a software-pipelined sequence: graph i runs
        the online phase of schedules[i] on triple slot i % 2 and deals
        next_schedules[i] into the other slot.  Replay the graphs in order, after
        deal(schedules[0], 0, join=True); stream order between replays orders each step's
        online phase after the dealing of the step before.  x is the input buffer
        the graphs read, or a list of buffers (graph i reads x[i % len(x)], so
        that the next step's input can be uploaded while a step runs).  Returns a
        list of (graph, revealed output) pairs."""
        xs = x if isinstance(x, (list, tuple)) else [x]
        out = []
        main = torch.cuda.current_stream()
        cs = torch.cuda.Stream(device=self.device)
        cs.wait_stream(main)
        with torch.cuda.stream(cs):
            for i, (sched, nxt) in enumerate(zip(schedules, next_schedules)):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cs):
                    y = self.reveal(self.forward_pipelined(xs[i % len(xs)], sched, i % 2, nxt,
                                                           wait_dealer=False))
                out.append((g, y))
        main.wait_stream(cs)
        return out
