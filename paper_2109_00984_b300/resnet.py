"""Private inference of a ResNet-18-shaped CNN as a sequence of library calls.

Two parties; the model owner (party 1) shares the weights once, the data owner
(party 0) shares each batch of images.  Per layer, the dealer calls produce
the material and the online calls consume it:
  convolution / linear:  ttp_conv2d_triple / ttp_matmul_triple, then
                         beaver_conv2d / beaver_matmul with fused truncation
  ReLU:                  ttp_and_triples, ttp_b2a_bits, ttp_mul_triple, private_relu
  residual connection:   add (local)
  3x3/2 max pool:        window_taps, then per tree level sub, one private_relu
                         over all pairs of the level, add (max(a,b) = b + ReLU(a-b))
  global average pool:   global_avgpool (local sum, floor division by H*W)
Material op_ids follow the schedule: a layer op with id `op` uses op (triple /
AND triples), op+1 (B2A bits), op+2 (ReLU's elementwise triple), op+3 (A2B
masks).  With fused_relu (the default) each ReLU is one private_relu_fused
call regenerating that material in registers (bit-identical results).
With overlap_dealer (the default) all convolution / linear triples of a forward
are dealt first on a second stream, which runs ahead of the online phase (the
dealer depends on shapes and op ids only); each online product waits on the
event recorded after its triple.
"""
import torch

from . import api


class PrivateResNet18:
    def __init__(self, weights, layers, schedule, algo=api.AUTO, frac_bits=16, device="cuda",
                 fused_relu=True, overlap_dealer=True, prepare_weights=False):
        self.P = 2
        self.fused_relu = fused_relu
        # With prepare_weights (limb engine, fused ReLU) the dealer also does each
        # convolution's input-independent half (F = W - B opened, the weight-side
        # and im2col(A_p) digit planes) right after its triple.
        self.prepare = prepare_weights and fused_relu and algo != api.PLAIN
        self.overlap_dealer = overlap_dealer
        # Online phase on a high-priority stream, dealer on a low-priority one.
        self.dealer_stream = torch.cuda.Stream(device=device, priority=0) if overlap_dealer \
            else None
        self.online_stream = torch.cuda.Stream(device=device, priority=-5) if overlap_dealer \
            else None
        self.dealer_ws = torch.empty(1, dtype=torch.uint8, device=device)
        self.layers = layers
        self.algo = algo
        self.frac_bits = frac_bits
        self.device = device
        self.seed = schedule["seed"]
        self.W = {}
        for i, name in enumerate(sorted(weights)):
            wt = torch.as_tensor(weights[name], dtype=torch.float64, device=device).contiguous()
            self.W[name] = api.ring_share(wt, self.P, 1, self.seed, schedule["weight_base"] + i,
                                          frac_bits)
        self.ws = torch.empty(1, dtype=torch.uint8, device=device)
        self._triples = {}

    def _ws(self, nbytes):
        if self.ws.numel() < nbytes:
            self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.ws

    def _dealer_ws(self, nbytes):
        if self.dealer_ws.numel() < nbytes:
            self.dealer_ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.dealer_ws

    # ---- dealer: convolution / linear triples ---------------------------------------
    def _deal_conv(self, d, op, ws):
        return api.ttp_conv2d_triple(self.P, d, self.seed, op, self.algo, device=self.device, ws=ws)

    def _deal_all(self, x_shape, schedule):
        """Walk the network's shapes and deal every conv / FC triple in order;
        the triples of consecutive same-shaped convolutions are dealt in one
        batched call (one GEMM launch for their products on the limb engine)."""
        ops = schedule["ops"]
        triples = {}
        N, _, H, W = x_shape
        C = 3
        pending = []   # (key, desc) of consecutive convolutions with one output shape

        def flush():
            if not pending:
                return
            descs = [dd for _, dd in pending]
            keys = [k for k, _ in pending]
            if len(keys) == 1:
                ws = self._dealer_ws(api.conv2d_triple_workspace_size(self.P, descs[0], self.algo))
                got = [self._deal_conv(descs[0], ops[keys[0]], ws)]
            else:
                ws = self._dealer_ws(api.conv2d_triples_workspace_size(self.P, len(keys), descs,
                                                                       self.algo))
                got = api.ttp_conv2d_triples(self.P, descs, self.seed, [ops[k] for k in keys],
                                             self.algo, device=self.device, ws=ws)
            for k, dd, t in zip(keys, descs, got):
                triples[k] = t
                if self.prepare and api.conv2d_prep_size(self.P, dd) > 0:
                    triples[k + "#prep"] = api.beaver_conv2d_prepare(self.W[k], t[0], t[1], dd)
            ev = torch.cuda.Event()
            ev.record(torch.cuda.current_stream())
            for k in keys:
                triples[k + "#ev"] = ev
            pending.clear()

        def conv(name, cin, cout, k, stride, pad, h, w, key):
            d = api.conv_desc(N, cin, h, w, cout, k, k, stride, stride, pad, pad)
            d0 = pending[0][1] if pending else None
            if pending and (len(pending) == api.MAX_TRIPLE_BATCH or
                            (d.c_out, d.batch) != (d0.c_out, d0.batch) or
                            api.conv_out_hw(d) != api.conv_out_hw(d0)):
                flush()
            pending.append((key, d))
            return api.conv_out_hw(d)

        for layer in self.layers:
            kind, name = layer[0], layer[1]
            if kind == "conv":
                H, W = conv(name, layer[2], layer[3], layer[4], layer[5], layer[6], H, W, name)
                C = layer[3]
            elif kind == "maxpool":
                H = (H + 2 * layer[4] - layer[2]) // layer[3] + 1
                W = (W + 2 * layer[4] - layer[2]) // layer[3] + 1
            elif kind == "block":
                _, name, cin, cout, s = layer
                h1, w1 = conv(name, cin, cout, 3, s, 1, H, W, name + ".conv1")
                conv(name, cout, cout, 3, 1, 1, h1, w1, name + ".conv2")
                if s != 1 or cin != cout:
                    conv(name, cin, cout, 1, s, 0, H, W, name + ".down")
                H, W, C = h1, w1, cout
            elif kind == "fc":
                flush()
                cin, cout = layer[2], layer[3]
                triples[name] = api.ttp_matmul_triple(self.P, N, cout, cin, self.seed, ops[name],
                                                      self.algo, device=self.device)
                ev = torch.cuda.Event()
                ev.record(torch.cuda.current_stream())
                triples[name + "#ev"] = ev
        flush()
        return triples

    def _triple(self, key):
        t = self._triples.get(key)
        if t is None:
            return None
        main = torch.cuda.current_stream()
        main.wait_event(self._triples[key + "#ev"])
        for tensor in t:        # allocated on the dealer stream, consumed here
            tensor.record_stream(main)
        return t

    def _prep(self, key):
        """The prepared planes of convolution `key` (after _triple), or None."""
        prep = self._triples.get(key + "#prep") if key is not None else None
        if prep is not None:
            prep.record_stream(torch.cuda.current_stream())
        return prep

    # ---- layer operations ---------------------------------------------------------
    def conv(self, X, Wsh, stride, pad, op, key=None):
        P, N, Cin, H, W = X.shape
        Cout, _, k, _ = Wsh.shape[1:]
        d = api.conv_desc(N, Cin, H, W, Cout, k, k, stride, stride, pad, pad)
        trip = self._triple(key) if key is not None else None
        if trip is None:
            ws = self._ws(max(api.conv2d_workspace_size(P, d, self.algo),
                              api.conv2d_triple_workspace_size(P, d, self.algo)))
            trip = self._deal_conv(d, op, ws)
        A, B, C = trip
        prep = self._prep(key)
        if prep is not None:
            ws = self._ws(api.conv2d_workspace_size(P, d, api.LIMB))
            return api.beaver_conv2d_prepared(X, A, C, prep, d, self.frac_bits, ws=ws)
        ws = self._ws(api.conv2d_workspace_size(P, d, self.algo))
        return api.beaver_conv2d(X, Wsh, A, B, C, d, self.algo, self.frac_bits, ws=ws)

    def conv_relu(self, X, Wsh, stride, pad, op, relu_op, key=None, add=None):
        """A convolution whose output (plus `add`, a residual shortcut, if given)
        goes straight into a ReLU: one composite call (the ReLU kernel reduces the
        GEMM's split-K partial sums and adds the shortcut itself)."""
        if not self.fused_relu:
            Z = self.conv(X, Wsh, stride, pad, op, key)
            return self.relu(Z if add is None else api.add(Z, add), relu_op)
        P, N, Cin, H, W = X.shape
        Cout, _, k, _ = Wsh.shape[1:]
        d = api.conv_desc(N, Cin, H, W, Cout, k, k, stride, stride, pad, pad)
        trip = self._triple(key) if key is not None else None
        if trip is None:
            ws = self._ws(max(api.conv2d_workspace_size(P, d, self.algo),
                              api.conv2d_triple_workspace_size(P, d, self.algo)))
            trip = self._deal_conv(d, op, ws)
        A, B, C = trip
        prep = self._prep(key)
        if prep is not None:
            ws = self._ws(api.conv2d_workspace_size(P, d, api.LIMB))
            return api.beaver_conv2d_relu_prepared(X, A, C, prep, d, self.seed, relu_op,
                                                   self.frac_bits, ws=ws, add=add)
        ws = self._ws(api.conv2d_workspace_size(P, d, self.algo))
        return api.beaver_conv2d_relu(X, Wsh, A, B, C, d, self.seed, relu_op, self.algo,
                                      self.frac_bits, ws=ws, add=add)

    def relu(self, X, op):
        P = X.shape[0]
        flat = X.reshape(P, -1)
        n = flat.shape[1]
        if self.fused_relu:
            return api.private_relu_fused(flat, self.seed, op).view(X.shape)
        T = api.ttp_and_triples(P, n, self.seed, op, device=self.device)
        ra, rb = api.ttp_b2a_bits(P, n, self.seed, op + 1, device=self.device)
        MT = torch.empty((3, P, n), dtype=torch.int64, device=self.device)
        api.ttp_mul_triple(P, n, self.seed, op + 2, out=(MT[0], MT[1], MT[2]))
        return api.private_relu(flat, T, ra, rb, MT, self.seed, op + 3).view(X.shape)

    def maxpool(self, X, k, stride, pad, ops):
        P = X.shape[0]
        taps = api.window_taps(X, k, stride, pad)
        shape = taps.shape[1:]
        vals = [taps[t].reshape(P, -1) for t in range(taps.shape[0])]
        n = vals[0].shape[1]
        level = 0
        while len(vals) > 1:
            npairs = len(vals) // 2
            if self.fused_relu and n % 4 == 0:
                # pair i of the level: b + ReLU(a - b) in one kernel, the ReLU's
                # material that of elements i n .. of the level's batched ReLU
                new = [api.private_max_fused(vals[2 * i], vals[2 * i + 1], self.seed,
                                             ops[level], elem_offset=i * n)
                       for i in range(npairs)]
                if len(vals) % 2:
                    new.append(vals[-1])
                vals = new
                level += 1
                continue
            D = torch.empty((P, npairs, n), dtype=torch.int64, device=self.device)
            for i in range(npairs):
                api.sub(vals[2 * i], vals[2 * i + 1], out=D[:, i])
            R = self.relu(D.view(P, npairs * n), ops[level]).view(P, npairs, n)
            new = [api.add(vals[2 * i + 1], R[:, i]) for i in range(npairs)]
            if len(vals) % 2:
                new.append(vals[-1])
            vals = new
            level += 1
        return vals[0].reshape(shape)

    def fc(self, X, Wsh, op, key=None):
        P, N, Cin = X.shape
        Cout = Wsh.shape[2]
        trip = self._triple(key) if key is not None else None
        if trip is None:
            trip = api.ttp_matmul_triple(P, N, Cout, Cin, self.seed, op, self.algo,
                                         device=self.device)
        A, B, C = trip
        return api.beaver_matmul(X, Wsh, A, B, C, self.algo, self.frac_bits)

    # ---- forward ----------------------------------------------------------------------
    def forward(self, x, schedule):
        """x: float64 CUDA images (N, 3, H, W).  Returns logit shares [2, N, classes]."""
        self._triples = {}
        if self.overlap_dealer:
            main = torch.cuda.current_stream()
            ds = self.dealer_stream
            ds.wait_stream(main)
            with torch.cuda.stream(ds):
                self._triples = self._deal_all(tuple(x.shape), schedule)
            on = self.online_stream
            on.wait_stream(main)
            with torch.cuda.stream(on):
                X = self._online(x, schedule)
                X.record_stream(main)
            main.wait_stream(on)
            return X
        return self._online(x, schedule)

    def _online(self, x, schedule):
        ops = schedule["ops"]
        X = api.ring_share(x, self.P, 0, self.seed, ops["input"], self.frac_bits)
        fused_next = False
        for li, layer in enumerate(self.layers):
            kind, name = layer[0], layer[1]
            if kind == "conv":
                nxt = self.layers[li + 1] if li + 1 < len(self.layers) else None
                if nxt is not None and nxt[0] == "relu":   # conv then ReLU: one call
                    X = self.conv_relu(X, self.W[name], layer[5], layer[6], ops[name],
                                       ops[nxt[1]], name)
                    fused_next = True
                else:
                    X = self.conv(X, self.W[name], layer[5], layer[6], ops[name], name)
            elif kind == "relu":
                if not fused_next:
                    X = self.relu(X, ops[name])
                fused_next = False
            elif kind == "maxpool":
                X = self.maxpool(X, layer[2], layer[3], layer[4],
                                 [ops[f"{name}.{l}"] for l in range(4)])
            elif kind == "block":
                _, name, cin, cout, s = layer
                Y = self.conv_relu(X, self.W[name + ".conv1"], s, 1, ops[name + ".conv1"],
                                   ops[name + ".relu1"], name + ".conv1")
                if s != 1 or cin != cout:
                    S = self.conv(X, self.W[name + ".down"], s, 0, ops[name + ".down"],
                                  name + ".down")
                else:
                    S = X
                # second convolution, shortcut and ReLU in one composite call
                X = self.conv_relu(Y, self.W[name + ".conv2"], 1, 1, ops[name + ".conv2"],
                                   ops[name + ".relu2"], name + ".conv2", add=S)
            elif kind == "avgpool":
                X = api.global_avgpool(X)
            elif kind == "fc":
                X = self.fc(X, self.W[name], ops[name], name)
        self._triples = {}
        return X

    def reveal(self, shares):
        _, real = api.reveal(shares, self.frac_bits, ring=False, real=True)
        return real

    def capture(self, x, schedules):
        """One CUDA graph per schedule of a whole private forward + reveal (both
        streams, dealer included); x is the device input buffer the graphs read.
        Returns a list of (graph, revealed logits) pairs."""
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
