// Binary shares for two parties: A2B with a Kogge-Stone adder, and the fused
// private ReLU = Beaver(x, B2A(MSB(A2B(-x)))) (§5.2 "Comparators", App.
// D.1.2-D.1.4, Alg. 2).  One kernel, one pass: every opening (the 12 AND
// gates' eps/delta, the B2A bit z, the Beaver E/F) is an XOR/sum of the two
// parties' registers.  Each thread owns 4 consecutive elements, i.e. one
// Philox block of each binary zero-share stream.
#include "common.cuh"
#include "host.hpp"
#include "fused.cuh"
#include "gemm.hpp"

namespace mpc {

namespace {

constexpr int kThreads = 256;


struct Pair {  // the two parties' shares of 4 elements
  Quad s[2];
};

// Secret AND of binary-shared x, y with gate g's triple; T is [gates][3][2][n].
__device__ __forceinline__ Pair and_gate(const Pair& x, const Pair& y, const u64* __restrict__ T,
                                         int g, i64 n, i64 i0) {
  const u64* base = T + (i64)g * 6 * n;
  const Quad a0 = load4(base + 0 * n, i0, n), a1 = load4(base + 1 * n, i0, n);
  const Quad b0 = load4(base + 2 * n, i0, n), b1 = load4(base + 3 * n, i0, n);
  const Quad c0 = load4(base + 4 * n, i0, n), c1 = load4(base + 5 * n, i0, n);
  Pair z;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const u64 eps = x.s[0].v[j] ^ a0.v[j] ^ x.s[1].v[j] ^ a1.v[j];
    const u64 del = y.s[0].v[j] ^ b0.v[j] ^ y.s[1].v[j] ^ b1.v[j];
    z.s[0].v[j] = c0.v[j] ^ (eps & b0.v[j]) ^ (a0.v[j] & del) ^ (eps & del);
    z.s[1].v[j] = c1.v[j] ^ (eps & b1.v[j]) ^ (a1.v[j] & del);
  }
  return z;
}

// Where an AND gate's triple comes from: loaded from the dealer's array T
// [gates][3][2][n], or regenerated in registers from the dealer's own streams
// (seed, op_id of the AND material): a_p = AND_A(g, p), b_p = AND_B(g, p),
// c_0 = AND_C(g, 0), c_1 = ((a_0 ^ a_1) & (b_0 ^ b_1)) ^ c_0 -- exactly what
// mpc_ttp_and_triples writes, so both give bit-identical results.
struct TripleSrc {
  const u64* T;  // loaded when non-null
  u64 seed, op_and;
  i64 blk;       // Philox block = element quad index
};

template <bool kGen>
__device__ __forceinline__ Pair and_gate_src(const Pair& x, const Pair& y, const TripleSrc& src,
                                             int g, i64 n, i64 i0) {
  if (!kGen) return and_gate(x, y, src.T, g, n, i0);
  const u64x4 a0 = prg_block(src.seed, src.op_and, stream_word2(MPC_ROLE_AND_A, g, 0), src.blk);
  const u64x4 a1 = prg_block(src.seed, src.op_and, stream_word2(MPC_ROLE_AND_A, g, 1), src.blk);
  const u64x4 b0 = prg_block(src.seed, src.op_and, stream_word2(MPC_ROLE_AND_B, g, 0), src.blk);
  const u64x4 b1 = prg_block(src.seed, src.op_and, stream_word2(MPC_ROLE_AND_B, g, 1), src.blk);
  const u64x4 c0 = prg_block(src.seed, src.op_and, stream_word2(MPC_ROLE_AND_C, g, 0), src.blk);
  Pair z;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const u64 c1 = ((a0.v[j] ^ a1.v[j]) & (b0.v[j] ^ b1.v[j])) ^ c0.v[j];
    const u64 eps = x.s[0].v[j] ^ a0.v[j] ^ x.s[1].v[j] ^ a1.v[j];
    const u64 del = y.s[0].v[j] ^ b0.v[j] ^ y.s[1].v[j] ^ b1.v[j];
    z.s[0].v[j] = c0.v[j] ^ (eps & b0.v[j]) ^ (a0.v[j] & del) ^ (eps & del);
    z.s[1].v[j] = c1 ^ (eps & b1.v[j]) ^ (a1.v[j] & del);
  }
  return z;
}

__device__ __forceinline__ Pair shl(const Pair& x, int d) {
  Pair o;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < 4; ++j) o.s[p].v[j] = x.s[p].v[j] << d;
  return o;
}

__device__ __forceinline__ Pair xr(const Pair& x, const Pair& y) {
  Pair o;
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int j = 0; j < 4; ++j) o.s[p].v[j] = x.s[p].v[j] ^ y.s[p].v[j];
  return o;
}

// A2B of arithmetic shares y (already negated for the comparator): binary-share
// each party's share with the ZERO_BIN streams, then Kogge-Stone add.
template <bool kGen>
__device__ __forceinline__ Pair a2b_block(const Pair& y, const TripleSrc& src, i64 n, i64 i0,
                                          i64 t, u64 seed, u64 op_id) {
  // M_{q,p}: ZERO_BIN stream of owner q, party p.
  const u64x4 m00 = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_BIN, 0, 0), t);
  const u64x4 m01 = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_BIN, 0, 1), t);
  const u64x4 m10 = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_BIN, 1, 0), t);
  const u64x4 m11 = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_BIN, 1, 1), t);
  // Party p holds M_{q,p} ^ M_{q,(p-1) mod 2} ^ [p == q] y_q.
  Pair u, v;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    u.s[0].v[j] = m00.v[j] ^ m01.v[j] ^ y.s[0].v[j];
    u.s[1].v[j] = m01.v[j] ^ m00.v[j];
    v.s[0].v[j] = m10.v[j] ^ m11.v[j];
    v.s[1].v[j] = m11.v[j] ^ m10.v[j] ^ y.s[1].v[j];
  }
  int gate = 0;
  Pair G = and_gate_src<kGen>(u, v, src, gate++, n, i0);
  Pair Pp = xr(u, v);
  const Pair P0 = Pp;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int d = 1 << r;  // 1, 2, 4, 8, 16, 32
    const Pair Gn = xr(G, and_gate_src<kGen>(Pp, shl(G, d), src, gate++, n, i0));
    if (d < 32) Pp = and_gate_src<kGen>(Pp, shl(Pp, d), src, gate++, n, i0);
    G = Gn;
  }
  return xr(P0, shl(G, 1));
}

__global__ void __launch_bounds__(kThreads) a2b_kernel(i64 n, const u64* __restrict__ X,
                                                       u64* __restrict__ Bout,
                                                       const u64* __restrict__ T, u64 seed,
                                                       u64 op_id) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Pair x;
    x.s[0] = load4(X, i0, n);
    x.s[1] = load4(X + n, i0, n);
    const Pair b = a2b_block<false>(x, TripleSrc{T, 0, 0, t}, n, i0, t, seed, op_id);
    store4(Bout, i0, n, b.s[0]);
    store4(Bout + n, i0, n, b.s[1]);
  }
}

// Private ReLU for two parties.  kGen = false: the material is read from the
// dealer's arrays.  kGen = true (fused dealer): it is regenerated in registers
// from the dealer's streams with op ids op_id (AND triples), op_id + 1 (B2A
// pairs), op_id + 2 (elementwise triple), and the A2B masks use op_id + 3 --
// the same words the separate dealer calls would have written.
template <bool kGen>
__global__ void __launch_bounds__(kThreads) relu_kernel(i64 n, const u64* X, u64* Y,
                                                        const u64* __restrict__ T,
                                                        const u64* __restrict__ r_arith,
                                                        const u64* __restrict__ r_bin,
                                                        const u64* __restrict__ MA,
                                                        const u64* __restrict__ MB,
                                                        const u64* __restrict__ MC, u64 seed,
                                                        u64 op_id) {
  const i64 nblk = ceil_div(n, 4);
  const i64 nw = ceil_div(n, 64);
  const u64 op_mask = kGen ? op_id + 3 : op_id;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Pair x, neg;
    x.s[0] = load4(X, i0, n);
    x.s[1] = load4(X + n, i0, n);
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int j = 0; j < 4; ++j) neg.s[p].v[j] = 0ull - x.s[p].v[j];
    // [x > 0] = [(0 - x) < 0]: sign bit of A2B(-x).
    const Pair sb = a2b_block<kGen>(neg, TripleSrc{T, seed, op_id, t}, n, i0, t, seed, op_mask);
    // B2A (Alg. 2): z = reveal(<b> ^ <r>), [b]_p = [r]_p - 2 z [r]_p + [p = 0] z.
    Quad ra0, ra1;
    u64 rbits;  // bit j = <r>_0 ^ <r>_1 of element i0 + j
    if (kGen) {
      const u64x4 r = prg_block(seed, op_id + 1, stream_word2(MPC_ROLE_B2A_R, 0, MPC_TTP_PARTY), t);
      const u64x4 rb = prg_block(seed, op_id + 1, stream_word2(MPC_ROLE_B2A_BIN, 0, 0), t);
      const u64x4 rr = prg_block(seed, op_id + 1, stream_word2(MPC_ROLE_B2A_ARITH, 0, 0), t);
      rbits = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // <r>_1 = r ^ <r>_0, so <r>_0 ^ <r>_1 = r; [r]_1 = r - [r]_0.
        rbits |= (r.v[j] & 1ull) << j;
        ra0.v[j] = rr.v[j];
        ra1.v[j] = (r.v[j] & 1ull) - rr.v[j];
      }
    } else {
      const int sh = (int)(i0 & 63);
      rbits = (r_bin[i0 >> 6] >> sh) ^ (r_bin[nw + (i0 >> 6)] >> sh);
      ra0 = load4(r_arith, i0, n);
      ra1 = load4(r_arith + n, i0, n);
    }
    Pair bit;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 z = ((sb.s[0].v[j] ^ sb.s[1].v[j]) >> 63) ^ ((rbits >> j) & 1ull);
      bit.s[0].v[j] = ra0.v[j] - 2ull * z * ra0.v[j] + z;
      bit.s[1].v[j] = ra1.v[j] - 2ull * z * ra1.v[j];
    }
    // Beaver product x * [b] (no truncation: the mask is an unscaled 0/1).
    Quad A0, A1, B0, B1, C0, C1;
    if (kGen) {
      const u64x4 a0 = prg_block(seed, op_id + 2, stream_word2(MPC_ROLE_TRIPLE_A, 0, 0), t);
      const u64x4 a1 = prg_block(seed, op_id + 2, stream_word2(MPC_ROLE_TRIPLE_A, 0, 1), t);
      const u64x4 b0 = prg_block(seed, op_id + 2, stream_word2(MPC_ROLE_TRIPLE_B, 0, 0), t);
      const u64x4 b1 = prg_block(seed, op_id + 2, stream_word2(MPC_ROLE_TRIPLE_B, 0, 1), t);
      const u64x4 c0 = prg_block(seed, op_id + 2, stream_word2(MPC_ROLE_TRIPLE_C, 0, 0), t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        A0.v[j] = a0.v[j];
        A1.v[j] = a1.v[j];
        B0.v[j] = b0.v[j];
        B1.v[j] = b1.v[j];
        C0.v[j] = c0.v[j];
        C1.v[j] = (a0.v[j] + a1.v[j]) * (b0.v[j] + b1.v[j]) - c0.v[j];
      }
    } else {
      A0 = load4(MA, i0, n);
      A1 = load4(MA + n, i0, n);
      B0 = load4(MB, i0, n);
      B1 = load4(MB + n, i0, n);
      C0 = load4(MC, i0, n);
      C1 = load4(MC + n, i0, n);
    }
    Quad y0, y1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 E = (x.s[0].v[j] - A0.v[j]) + (x.s[1].v[j] - A1.v[j]);
      const u64 F = (bit.s[0].v[j] - B0.v[j]) + (bit.s[1].v[j] - B1.v[j]);
      y0.v[j] = C0.v[j] + E * B0.v[j] + A0.v[j] * F + E * F;
      y1.v[j] = C1.v[j] + E * B1.v[j] + A1.v[j] * F;
    }
    store4(Y, i0, n, y0);
    store4(Y + n, i0, n, y1);
  }
}

// [x < 0] for two parties: A2B of x (no negation), sign bit, B2A (Alg. 2).
__global__ void __launch_bounds__(kThreads) ltz_kernel(i64 n, const u64* X, u64* Out,
                                                       const u64* __restrict__ T,
                                                       const u64* __restrict__ r_arith,
                                                       const u64* __restrict__ r_bin, u64 seed,
                                                       u64 op_id) {
  const i64 nblk = ceil_div(n, 4);
  const i64 nw = ceil_div(n, 64);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Pair x;
    x.s[0] = load4(X, i0, n);
    x.s[1] = load4(X + n, i0, n);
    const Pair sb = a2b_block<false>(x, TripleSrc{T, 0, 0, t}, n, i0, t, seed, op_id);
    const int sh = (int)(i0 & 63);
    const u64 rbits = (r_bin[i0 >> 6] >> sh) ^ (r_bin[nw + (i0 >> 6)] >> sh);
    const Quad ra0 = load4(r_arith, i0, n), ra1 = load4(r_arith + n, i0, n);
    Quad b0, b1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 z = ((sb.s[0].v[j] ^ sb.s[1].v[j]) >> 63) ^ ((rbits >> j) & 1ull);
      b0.v[j] = ra0.v[j] - 2ull * z * ra0.v[j] + z;
      b1.v[j] = ra1.v[j] - 2ull * z * ra1.v[j];
    }
    store4(Out, i0, n, b0);
    store4(Out + n, i0, n, b1);
  }
}

// S (may be null): ReLU of X + S, the private addition of two sharings (local:
// each party adds its shares) folded into the load.  With max_mode, S + ReLU(X
// - S) = max(X, S) instead (the comparison of a max-pool tree, both local
// steps folded in).  blk_off: the dealer material of element i is that of
// element i + 4 blk_off of a longer ReLU (a slice of a batched comparison).
__global__ void __launch_bounds__(256, 3) relu_fused_quad_kernel(i64 n, const u64* X,
                                                              const u64* S, u64* Y, u64 seed,
                                                              u64 op, int max_mode,
                                                              i64 blk_off) {
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(n, (i64)blockDim.x) * blockDim.x;  // uniform trip count per block
  const int j = threadIdx.x & 3;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < npad; i += stride) {
    const bool valid = i < n;
    const i64 blk = (i >> 2) + blk_off;
    Sh2 x{{valid ? X[i] : 0ull, valid ? X[n + i] : 0ull}};
    Sh2 s{{0ull, 0ull}};
    if (S && valid) {
      s.v[0] = S[i];
      s.v[1] = S[n + i];
    }
    if (max_mode) {
      x.v[0] -= s.v[0];
      x.v[1] -= s.v[1];
    } else {
      x.v[0] += s.v[0];
      x.v[1] += s.v[1];
    }
    Sh2 y = relu_quad(x, seed, op, blk, j);
    if (max_mode) {
      y.v[0] += s.v[0];
      y.v[1] += s.v[1];
    }
    if (valid) {
      Y[i] = y.v[0];
      Y[n + i] = y.v[1];
    }
  }
}

// The fused ReLU of a two-party GEMM job set's output, reduced on the fly: x_p
// of output index i = trunc(C_p[i] + sum_s partial[s][p][row][col]) with
// (row, col) the GEMM position of i (inverse of gemm_out_index), or Z_p[i]
// when the job set was not split.  Same grid and quad layout as
// relu_fused_quad_kernel.
__global__ void __launch_bounds__(256, 3) relu_gemm_quad_kernel(const GemmArgs g, u64* Y,
                                                             u64 seed, u64 op,
                                                             const u64* __restrict__ S) {
  const i64 n = g.M * g.N;
  const i64 stride = (i64)gridDim.x * blockDim.x;
  const i64 npad = ceil_div(n, (i64)blockDim.x) * blockDim.x;  // uniform trip count per block
  const int j = threadIdx.x & 3;
  const i64 sstride = (i64)g.njobs * n;
  for (i64 i = (i64)blockIdx.x * blockDim.x + threadIdx.x; i - threadIdx.x < npad; i += stride) {
    const bool valid = i < n;
    Sh2 x{{0ull, 0ull}};
    if (valid) {
      if (g.splits > 1) {
        i64 row, col;
        if (g.hw_out) {  // i = (b M + row) hw + pos, col = b hw + pos
          const i64 q = i / g.hw_out, pos = i - q * g.hw_out;
          const i64 b = q / g.M;
          row = q - b * g.M;
          col = b * g.hw_out + pos;
        } else {
          row = i / g.N;
          col = i - row * g.N;
        }
        const u64* part = g.partial + row * g.N + col;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          u64 acc = g.jobs[p].C ? g.jobs[p].C[i] : 0ull;
          for (int sp = 0; sp < g.splits; ++sp) acc += part[sp * sstride + p * n];
          x.v[p] = g.trunc_bits > 0 ? sar(acc, g.trunc_bits) : acc;
        }
      } else {
        x.v[0] = g.jobs[0].Z[i];
        x.v[1] = g.jobs[1].Z[i];
      }
      if (S) {  // a residual sum, added to the truncated product
        x.v[0] += S[i];
        x.v[1] += S[n + i];
      }
    }
    const Sh2 y = relu_quad(x, seed, op, i >> 2, j);
    if (valid) {
      Y[i] = y.v[0];
      Y[n + i] = y.v[1];
    }
  }
}

// ---- any number of parties: a tree of adders (one element per thread) ---------------
// Adders are numbered level by level, left to right; adder a uses gates 12a..12a+11
// of T [12 (P-1)][3][P][n].
template <int P>
struct Shares {
  u64 v[P];
};

template <int P>
__device__ __forceinline__ Shares<P> and_gate_p(const Shares<P>& x, const Shares<P>& y,
                                               const u64* __restrict__ T, int g, i64 n, i64 i) {
  const u64* base = T + (i64)g * 3 * P * n + i;
  u64 eps = 0, del = 0;
  u64 a[P], b[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    a[p] = base[(i64)p * n];
    b[p] = base[(i64)(P + p) * n];
    eps ^= x.v[p] ^ a[p];
    del ^= y.v[p] ^ b[p];
  }
  Shares<P> z;
#pragma unroll
  for (int p = 0; p < P; ++p)
    z.v[p] = base[(i64)(2 * P + p) * n] ^ (eps & b[p]) ^ (a[p] & del) ^ (p == 0 ? (eps & del) : 0ull);
  return z;
}

template <int P>
__device__ __forceinline__ Shares<P> ks_add_p(const Shares<P>& x, const Shares<P>& y,
                                             const u64* __restrict__ T, int adder, i64 n, i64 i) {
  int gate = adder * MPC_KS_GATES;
  Shares<P> G = and_gate_p<P>(x, y, T, gate++, n, i);
  Shares<P> Pp, P0;
#pragma unroll
  for (int p = 0; p < P; ++p) Pp.v[p] = P0.v[p] = x.v[p] ^ y.v[p];
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int d = 1 << r;
    Shares<P> Gs, Ps;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Gs.v[p] = G.v[p] << d;
      Ps.v[p] = Pp.v[p] << d;
    }
    const Shares<P> t = and_gate_p<P>(Pp, Gs, T, gate++, n, i);
    if (d < 32) Pp = and_gate_p<P>(Pp, Ps, T, gate++, n, i);
#pragma unroll
    for (int p = 0; p < P; ++p) G.v[p] ^= t.v[p];
  }
  Shares<P> out;
#pragma unroll
  for (int p = 0; p < P; ++p) out.v[p] = P0.v[p] ^ (G.v[p] << 1);
  return out;
}

// A2B of arithmetic shares y (one element): binary-share every party's share,
// then add with the tree.
template <int P>
__device__ __forceinline__ Shares<P> a2b_tree(const Shares<P>& y, const u64* __restrict__ T,
                                             i64 n, i64 i, u64 seed, u64 op_id) {
  const i64 blk = i >> 2;
  const int w = (int)(i & 3);
  Shares<P> vals[P];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    u64 m[P];
#pragma unroll
    for (int p = 0; p < P; ++p)
      m[p] = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_BIN, q, p), blk).v[w];
#pragma unroll
    for (int p = 0; p < P; ++p)
      vals[q].v[p] = m[p] ^ m[(p + P - 1) % P] ^ (p == q ? y.v[q] : 0ull);
  }
  int count = P, adder = 0;
#pragma unroll
  for (int level = 0; level < 3; ++level) {
    if (count <= 1) break;
    int out = 0;
#pragma unroll
    for (int j = 0; j + 1 < P; j += 2) {
      if (j + 1 < count) vals[out++] = ks_add_p<P>(vals[j], vals[j + 1], T, adder++, n, i);
    }
    if (count & 1) vals[out++] = vals[count - 1];
    count = out;
  }
  return vals[0];
}

template <int P>
__global__ void __launch_bounds__(128) a2b_tree_kernel(i64 n, const u64* __restrict__ X,
                                                       u64* __restrict__ Bout,
                                                       const u64* __restrict__ T, u64 seed,
                                                       u64 op_id) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    Shares<P> y;
#pragma unroll
    for (int p = 0; p < P; ++p) y.v[p] = X[(i64)p * n + i];
    const Shares<P> b = a2b_tree<P>(y, T, n, i, seed, op_id);
#pragma unroll
    for (int p = 0; p < P; ++p) Bout[(i64)p * n + i] = b.v[p];
  }
}

template <int P>
__global__ void __launch_bounds__(128) relu_tree_kernel(i64 n, const u64* X, u64* Y,
                                                        const u64* __restrict__ T,
                                                        const u64* __restrict__ r_arith,
                                                        const u64* __restrict__ r_bin,
                                                        const u64* __restrict__ MA,
                                                        const u64* __restrict__ MB,
                                                        const u64* __restrict__ MC, u64 seed,
                                                        u64 op_id) {
  const i64 nw = ceil_div(n, 64);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    Shares<P> x, neg;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      x.v[p] = X[(i64)p * n + i];
      neg.v[p] = 0ull - x.v[p];
    }
    const Shares<P> sb = a2b_tree<P>(neg, T, n, i, seed, op_id);
    // B2A (Alg. 2) of the sign bit, then the Beaver product with the 0/1 mask.
    u64 z = 0;
#pragma unroll
    for (int p = 0; p < P; ++p)
      z ^= (sb.v[p] >> 63) ^ ((r_bin[(i64)p * nw + (i >> 6)] >> (i & 63)) & 1ull);
    u64 E = 0, F = 0, bit[P], A[P], B[P];
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const u64 ra = r_arith[(i64)p * n + i];
      bit[p] = ra - 2ull * z * ra + (p == 0 ? z : 0ull);
      A[p] = MA[(i64)p * n + i];
      B[p] = MB[(i64)p * n + i];
      E += x.v[p] - A[p];
      F += bit[p] - B[p];
    }
#pragma unroll
    for (int p = 0; p < P; ++p)
      Y[(i64)p * n + i] = MC[(i64)p * n + i] + E * B[p] + A[p] * F +
                          (p == 0 ? E * F : 0ull);
  }
}

template <int P>
__global__ void __launch_bounds__(128) ltz_tree_kernel(i64 n, const u64* X, u64* Out,
                                                       const u64* __restrict__ T,
                                                       const u64* __restrict__ r_arith,
                                                       const u64* __restrict__ r_bin, u64 seed,
                                                       u64 op_id) {
  const i64 nw = ceil_div(n, 64);
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    Shares<P> x;
#pragma unroll
    for (int p = 0; p < P; ++p) x.v[p] = X[(i64)p * n + i];
    const Shares<P> sb = a2b_tree<P>(x, T, n, i, seed, op_id);
    u64 z = 0;
#pragma unroll
    for (int p = 0; p < P; ++p)
      z ^= (sb.v[p] >> 63) ^ ((r_bin[(i64)p * nw + (i >> 6)] >> (i & 63)) & 1ull);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const u64 ra = r_arith[(i64)p * n + i];
      Out[(i64)p * n + i] = ra - 2ull * z * ra + (p == 0 ? z : 0ull);
    }
  }
}

template <int P>
void launch_ltz_tree(i64 n, const u64* X, u64* Out, const u64* T, const u64* ra, const u64* rb,
                     u64 seed, u64 op, cudaStream_t s) {
  ltz_tree_kernel<P><<<grid_for(n, 128), 128, 0, s>>>(n, X, Out, T, ra, rb, seed, op);
}

template <int P>
void launch_a2b_tree(i64 n, const u64* X, u64* B, const u64* T, u64 seed, u64 op, cudaStream_t s) {
  a2b_tree_kernel<P><<<grid_for(n, 128), 128, 0, s>>>(n, X, B, T, seed, op);
}

template <int P>
void launch_relu_tree(i64 n, const u64* X, u64* Y, const u64* T, const u64* ra, const u64* rb,
                      const u64* MA, const u64* MB, const u64* MC, u64 seed, u64 op,
                      cudaStream_t s) {
  relu_tree_kernel<P><<<grid_for(n, 128), 128, 0, s>>>(n, X, Y, T, ra, rb, MA, MB, MC, seed, op);
}

// Rounds of the adder tree: 7 per level, ceil(log2 P) levels.
inline uint64_t a2b_rounds(int P) {
  int levels = 0;
  for (int c = P; c > 1; c = (c + 1) / 2) ++levels;
  return 7ull * levels;
}

#define MPC_DISPATCH_P3(P, FN, ...)      \
  switch (P) {                           \
    case 3: FN<3>(__VA_ARGS__); break;   \
    case 4: FN<4>(__VA_ARGS__); break;   \
    case 5: FN<5>(__VA_ARGS__); break;   \
    case 6: FN<6>(__VA_ARGS__); break;   \
    case 7: FN<7>(__VA_ARGS__); break;   \
    default: FN<8>(__VA_ARGS__); break;  \
  }

}  // namespace

int launch_relu_of_gemm(const GemmArgs& g, u64* Y, u64 seed, u64 op, cudaStream_t s,
                        const u64* S) {
  if (g.njobs != 2) return fail(MPC_EUNSUPPORTED, "fused ReLU of a GEMM needs two parties");
  const i64 n = g.M * g.N;
  if (n == 0) return MPC_OK;
  {
    KernelTimer timer("private_relu_fused", s);
    relu_gemm_quad_kernel<<<grid_for(n, 256, 148 * 8), 256, 0, s>>>(g, Y, seed, op, S);
    if (int rc = check_launch("private_relu_fused (of a GEMM)")) return rc;
  }
  stats_add(9, (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div(n, 8) + 16ull * n,
            (uint64_t)MPC_KS_GATES * n, (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n + 6ull * n, 0);
  return MPC_OK;
}

}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_a2b(int P, int64_t n, const uint64_t* arith, uint64_t* binary,
            const uint64_t* and_triples, uint64_t seed, uint64_t op_id, void* stream) {
  if (P == 1) return fail(MPC_EUNSUPPORTED, "A2B needs at least two parties");
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(arith && binary && and_triples, "null pointer");
  if (P > 2) {
    {
      KernelTimer timer("a2b", as_stream(stream));
      MPC_DISPATCH_P3(P, launch_a2b_tree, n, (const u64*)arith, (u64*)binary,
                      (const u64*)and_triples, seed, op_id, as_stream(stream));
    }
    int rc = check_launch("a2b (adder tree)");
    if (rc == MPC_OK)
      stats_add(a2b_rounds(P), (uint64_t)MPC_KS_GATES * (P - 1) * 16ull * n,
                (uint64_t)MPC_KS_GATES * (P - 1) * n, (uint64_t)MPC_KS_GATES * (P - 1) * 3ull * P * n,
                0);
    return rc;
  }
  int rc;
  {
    KernelTimer timer("a2b", as_stream(stream));
    a2b_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
        n, (const u64*)arith, (u64*)binary, (const u64*)and_triples, seed, op_id);
    rc = check_launch("a2b");
  }
  if (rc == MPC_OK)
    stats_add(7, (uint64_t)MPC_KS_GATES * 16ull * n, (uint64_t)MPC_KS_GATES * n,
              (uint64_t)MPC_KS_GATES * 6ull * n, 0);
  return rc;
}

int mpc_private_relu(int P, int64_t n, const uint64_t* X, uint64_t* Y,
                     const uint64_t* and_triples, const uint64_t* r_arith,
                     const uint64_t* r_bin, const uint64_t* mul_A, const uint64_t* mul_B,
                     const uint64_t* mul_C, uint64_t seed, uint64_t op_id, void* stream) {
  if (P == 1) return fail(MPC_EUNSUPPORTED, "private ReLU needs at least two parties");
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y && and_triples && r_arith && r_bin && mul_A && mul_B && mul_C,
              "null pointer");
  if (P > 2) {
    {
      KernelTimer timer("private_relu", as_stream(stream));
      MPC_DISPATCH_P3(P, launch_relu_tree, n, (const u64*)X, (u64*)Y, (const u64*)and_triples,
                      (const u64*)r_arith, (const u64*)r_bin, (const u64*)mul_A,
                      (const u64*)mul_B, (const u64*)mul_C, seed, op_id, as_stream(stream));
    }
    int rc = check_launch("private_relu (adder tree)");
    if (rc == MPC_OK)
      stats_add(a2b_rounds(P) + 2, (uint64_t)MPC_KS_GATES * (P - 1) * 16ull * n + 16ull * n,
                (uint64_t)MPC_KS_GATES * (P - 1) * n,
                (uint64_t)MPC_KS_GATES * (P - 1) * 3ull * P * n + 5ull * P * n, 0);
    return rc;
  }
  int rc;
  {
    KernelTimer timer("private_relu", as_stream(stream));
    relu_kernel<false><<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
        n, (const u64*)X, (u64*)Y, (const u64*)and_triples, (const u64*)r_arith,
        (const u64*)r_bin, (const u64*)mul_A, (const u64*)mul_B, (const u64*)mul_C, seed, op_id);
    rc = check_launch("private_relu");
  }
  if (rc == MPC_OK)
    stats_add(9, (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div(n, 8) + 16ull * n,
              (uint64_t)MPC_KS_GATES * n, (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n + 6ull * n,
              0);
  return rc;
}

int mpc_private_relu_fused(int P, int64_t n, const uint64_t* X, uint64_t* Y, uint64_t seed,
                           uint64_t op_id, void* stream) {
  return mpc_private_relu_fused_add(P, n, X, nullptr, Y, seed, op_id, stream);
}

int mpc_private_relu_fused_add(int P, int64_t n, const uint64_t* X, const uint64_t* S,
                               uint64_t* Y, uint64_t seed, uint64_t op_id, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "fused private ReLU supports P = 2 (got %d)", P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y, "null pointer");
  int rc;
  {
    KernelTimer timer("private_relu_fused", as_stream(stream));
    relu_fused_quad_kernel<<<grid_for(n, 256, 148 * 8), 256, 0, as_stream(stream)>>>(
        n, (const u64*)X, (const u64*)S, (u64*)Y, seed, op_id, 0, 0);
    rc = check_launch("private_relu_fused");
  }
  if (rc == MPC_OK)
    stats_add(9, (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div(n, 8) + 16ull * n,
              (uint64_t)MPC_KS_GATES * n, (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n + 6ull * n,
              0);
  return rc;
}

int mpc_private_max_fused(int P, int64_t n, const uint64_t* A, const uint64_t* B, uint64_t* Y,
                          uint64_t seed, uint64_t op_id, int64_t elem_offset, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "fused private max supports P = 2 (got %d)", P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(elem_offset >= 0 && elem_offset % 4 == 0,
              "element offset %lld is not a non-negative multiple of 4", (long long)elem_offset);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(A && B && Y, "null pointer");
  int rc;
  {
    KernelTimer timer("private_relu_fused", as_stream(stream));
    relu_fused_quad_kernel<<<grid_for(n, 256, 148 * 8), 256, 0, as_stream(stream)>>>(
        n, (const u64*)A, (const u64*)B, (u64*)Y, seed, op_id, 1, elem_offset / 4);
    rc = check_launch("private_max_fused");
  }
  // the slices of one batched comparison share its rounds: counted once, by
  // the slice at offset 0
  if (rc == MPC_OK)
    stats_add(elem_offset == 0 ? 9 : 0, (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div(n, 8) + 16ull * n,
              (uint64_t)MPC_KS_GATES * n, (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n + 6ull * n,
              0);
  return rc;
}

int mpc_ltz(int P, int64_t n, const uint64_t* X, uint64_t* out, const uint64_t* and_triples,
            const uint64_t* r_arith, const uint64_t* r_bin, uint64_t seed, uint64_t op_id,
            void* stream) {
  if (P == 1) return fail(MPC_EUNSUPPORTED, "comparison needs at least two parties");
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && out && and_triples && r_arith && r_bin, "null pointer");
  cudaStream_t s = as_stream(stream);
  if (P == 2) {
    ltz_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, s>>>(
        n, (const u64*)X, (u64*)out, (const u64*)and_triples, (const u64*)r_arith,
        (const u64*)r_bin, seed, op_id);
  } else {
    MPC_DISPATCH_P3(P, launch_ltz_tree, n, (const u64*)X, (u64*)out, (const u64*)and_triples,
                    (const u64*)r_arith, (const u64*)r_bin, seed, op_id, s);
  }
  int rc = check_launch("ltz");
  if (rc == MPC_OK)
    stats_add(a2b_rounds(P) + 1, (uint64_t)MPC_KS_GATES * (P - 1) * 16ull * n + ceil_div(n, 8),
              (uint64_t)MPC_KS_GATES * (P - 1) * n,
              (uint64_t)MPC_KS_GATES * (P - 1) * 3ull * P * n + 2ull * P * n, 0);
  return rc;
}

}  // extern "C"
