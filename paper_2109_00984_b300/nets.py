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
own workspace.
"""
import torch

from . import api


class PrivateConv1dStack:
    def __init__(self, weights, strides, pads, frames, batch=1, algo=api.PLAIN, frac_bits=16,
                 weight_ops=None, seed=1, device="cuda", fused_relu=True, overlap_dealer=True):
        self.P = 2
        self.fused_relu = fused_relu
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

    def _alloc(self):
        P, dev = self.P, self.device
        self.X0 = torch.empty((P,) + self.in_shape, dtype=torch.int64, device=dev)
        self.bufs = []
        ws_bytes = 0
        for d in self.descs:
            ho, wo = api.conv_out_hw(d)
            n = d.batch * d.c_out * ho * wo
            b = dict(
                A=torch.empty((P, d.batch, d.c_in, d.h, d.w), dtype=torch.int64, device=dev),
                B=torch.empty((P, d.c_out, d.c_in, d.kh, d.kw), dtype=torch.int64, device=dev),
                C=torch.empty((P, d.batch, d.c_out, ho, wo), dtype=torch.int64, device=dev),
                Z=torch.empty((P, d.batch, d.c_out, ho, wo), dtype=torch.int64, device=dev),
                Y=torch.empty((P, d.batch, d.c_out, ho, wo), dtype=torch.int64, device=dev),
                n=n,
            )
            ws_bytes = max(ws_bytes, api.conv2d_workspace_size(P, d, self.algo),
                           api.conv2d_triple_workspace_size(P, d, self.algo))
            if not self.fused_relu:
                b.update(T=torch.empty((api.KS_GATES, 3, P, n), dtype=torch.int64, device=dev),
                         ra=torch.empty((P, n), dtype=torch.int64, device=dev),
                         rb=torch.empty((P, (n + 63) // 64), dtype=torch.int64, device=dev),
                         MT=torch.empty((3, P, n), dtype=torch.int64, device=dev))
            self.bufs.append(b)
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

    def forward(self, x, schedule):
        """x: float64 CUDA tensor of the input shape. Returns output shares [P, ...]."""
        seed = schedule["seed"]
        main = torch.cuda.current_stream()
        ready = []
        if self.overlap_dealer:
            ds = self.dealer_stream
            ds.wait_stream(main)
            with torch.cuda.stream(ds):
                for l, (d, b) in enumerate(zip(self.descs, self.bufs)):
                    api.ttp_conv2d_triple(self.P, d, seed, schedule["layers"][l]["conv"], self.algo,
                                          out=(b["A"], b["B"], b["C"]), ws=self.dealer_ws)
                    ev = torch.cuda.Event()
                    ev.record(ds)
                    ready.append(ev)
        if self.overlap_dealer:
            on = self.online_stream
            on.wait_stream(main)
            with torch.cuda.stream(on):
                X = self._online(x, schedule, on, ready)
            main.wait_stream(on)
            return X
        return self._online(x, schedule, main, ready)

    def _online(self, x, schedule, main, ready):
        seed = schedule["seed"]
        api.ring_share(x, self.P, 0, seed, schedule["input_op"], self.frac_bits, out=self.X0)
        X = self.X0
        for l, (d, b) in enumerate(zip(self.descs, self.bufs)):
            ops = schedule["layers"][l]
            if self.overlap_dealer:
                main.wait_event(ready[l])
            else:
                api.ttp_conv2d_triple(self.P, d, seed, ops["conv"], self.algo,
                                      out=(b["A"], b["B"], b["C"]), ws=self.ws)
            api.beaver_conv2d(X, self.W[l], b["A"], b["B"], b["C"], d, self.algo,
                              trunc_bits=self.frac_bits, out=b["Z"], ws=self.ws)
            n = b["n"]
            if self.fused_relu:
                assert (ops["b2a"], ops["mul"], ops["relu"]) == (ops["and"] + 1, ops["and"] + 2,
                                                                 ops["and"] + 3)
                api.private_relu_fused(b["Z"], seed, ops["and"], out=b["Y"])
            else:
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
