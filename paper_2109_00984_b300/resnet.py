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
"""
import torch

from . import api


class PrivateResNet18:
    def __init__(self, weights, layers, schedule, algo=api.AUTO, frac_bits=16, device="cuda",
                 fused_relu=True):
        self.P = 2
        self.fused_relu = fused_relu
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

    def _ws(self, nbytes):
        if self.ws.numel() < nbytes:
            self.ws = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.ws

    # ---- layer operations ---------------------------------------------------------
    def conv(self, X, Wsh, stride, pad, op):
        P, N, Cin, H, W = X.shape
        Cout, _, k, _ = Wsh.shape[1:]
        d = api.conv_desc(N, Cin, H, W, Cout, k, k, stride, stride, pad, pad)
        ws = self._ws(max(api.conv2d_workspace_size(P, d, self.algo),
                          api.conv2d_triple_workspace_size(P, d, self.algo)))
        A, B, C = api.ttp_conv2d_triple(P, d, self.seed, op, self.algo, device=self.device, ws=ws)
        return api.beaver_conv2d(X, Wsh, A, B, C, d, self.algo, self.frac_bits, ws=ws)

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

    def fc(self, X, Wsh, op):
        P, N, Cin = X.shape
        Cout = Wsh.shape[2]
        A, B, C = api.ttp_matmul_triple(P, N, Cout, Cin, self.seed, op, self.algo,
                                        device=self.device)
        return api.beaver_matmul(X, Wsh, A, B, C, self.algo, self.frac_bits)

    # ---- forward ----------------------------------------------------------------------
    def forward(self, x, schedule):
        """x: float64 CUDA images (N, 3, H, W).  Returns logit shares [2, N, classes]."""
        ops = schedule["ops"]
        X = api.ring_share(x, self.P, 0, self.seed, ops["input"], self.frac_bits)
        for layer in self.layers:
            kind, name = layer[0], layer[1]
            if kind == "conv":
                X = self.conv(X, self.W[name], layer[5], layer[6], ops[name])
            elif kind == "relu":
                X = self.relu(X, ops[name])
            elif kind == "maxpool":
                X = self.maxpool(X, layer[2], layer[3], layer[4],
                                 [ops[f"{name}.{l}"] for l in range(4)])
            elif kind == "block":
                _, name, cin, cout, s = layer
                Y = self.conv(X, self.W[name + ".conv1"], s, 1, ops[name + ".conv1"])
                Y = self.relu(Y, ops[name + ".relu1"])
                Y = self.conv(Y, self.W[name + ".conv2"], 1, 1, ops[name + ".conv2"])
                if s != 1 or cin != cout:
                    S = self.conv(X, self.W[name + ".down"], s, 0, ops[name + ".down"])
                else:
                    S = X
                X = self.relu(api.add(Y, S), ops[name + ".relu2"])
            elif kind == "avgpool":
                X = api.global_avgpool(X)
            elif kind == "fc":
                X = self.fc(X, self.W[name], ops[name])
        return X

    def reveal(self, shares):
        _, real = api.reveal(shares, self.frac_bits, ring=False, real=True)
        return real
