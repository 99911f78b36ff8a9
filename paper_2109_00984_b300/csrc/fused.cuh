// Fused-dealer building blocks for two parties, one element per thread: Philox
// words of four streams shared across a quad of lanes, Boolean and arithmetic
// Beaver steps on register-held shares, [y < 0] (A2B, MSB, B2A) and ReLU.
// Every "opening" is a sum (or XOR) over the two shares held by the thread.
#pragma once

#include "common.cuh"

namespace mpc {

// ---- fused dealer, one element per thread ------------------------------------------------
// Lanes 4q..4q+3 hold four consecutive elements, i.e. one Philox block of every
// stream.  For a group of four streams each lane computes the block of one
// stream and the words are exchanged by shuffles, so every lane ends with its
// element's word of all four streams: the same Philox work as one block per
// four elements, with one element of protocol state per thread.
struct Quad4 {
  u64 w[4];  // word of this lane's element in streams 0..3 of the group
};

__device__ __forceinline__ Quad4 quad_gen(u64 seed, u64 op0, u64 w0, u64 op1, u64 w1, u64 op2,
                                          u64 w2, u64 op3, u64 w3, i64 blk, int j) {
  const u64 op = j == 0 ? op0 : j == 1 ? op1 : j == 2 ? op2 : op3;
  const u64 wd = j == 0 ? w0 : j == 1 ? w1 : j == 2 ? w2 : w3;
  const u64x4 b = prg_block(seed, op, wd, blk);
  // 4 x 4 transpose across the quad (lane j holds block j, wants word j of
  // blocks 0..3): two butterfly stages over lane bits 1 and 2, each swapping
  // the half of the words whose index bit differs from the lane bit.
  u64 a[4] = {b.v[0], b.v[1], b.v[2], b.v[3]};
#pragma unroll
  for (int m = 1; m <= 2; m <<= 1) {
    const bool hi = (j & m) != 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k & m) continue;
      const u64 t = __shfl_xor_sync(0xffffffffu, hi ? a[k] : a[k | m], m);
      if (hi)
        a[k] = t;
      else
        a[k | m] = t;
    }
  }
  Quad4 q;
#pragma unroll
  for (int s = 0; s < 4; ++s) q.w[s] = a[s];
  return q;
}

struct Sh2 {
  u64 v[2];
};

__device__ __forceinline__ Sh2 xr2(Sh2 a, Sh2 b) { return Sh2{{a.v[0] ^ b.v[0], a.v[1] ^ b.v[1]}}; }
__device__ __forceinline__ Sh2 shl2(Sh2 a, int d) { return Sh2{{a.v[0] << d, a.v[1] << d}}; }

// AND with a triple (a0, a1, b0, b1, c0), c1 = ((a0 ^ a1) & (b0 ^ b1)) ^ c0.
__device__ __forceinline__ Sh2 and2(Sh2 x, Sh2 y, const Quad4& ab, u64 c0) {
  const u64 a0 = ab.w[0], a1 = ab.w[1], b0 = ab.w[2], b1 = ab.w[3];
  const u64 c1 = ((a0 ^ a1) & (b0 ^ b1)) ^ c0;
  const u64 eps = x.v[0] ^ a0 ^ x.v[1] ^ a1;
  const u64 del = y.v[0] ^ b0 ^ y.v[1] ^ b1;
  return Sh2{{c0 ^ (eps & b0) ^ (a0 & del) ^ (eps & del), c1 ^ (eps & b1) ^ (a1 & del)}};
}

// [y < 0] as arithmetic 0/1 shares (Sections 5.2 "Comparators" and App. D.1.2):
// A2B of y with ZERO_BIN masks at op + 3, the Kogge-Stone adder with AND triples
// at op, MSB, B2A with the pair at op + 1 (Alg. 2).  The B2A group has a spare
// fourth stream; its word (stream (extra_op, extra_w2)) is returned in `extra`.
__device__ __forceinline__ Sh2 ltz_quad(Sh2 y, u64 seed, u64 op, i64 blk, int j, u64 extra_op,
                                        u64 extra_w2, u64& extra) {
  const u64 op_and = op, op_b2a = op + 1, op_mask = op + 3;
  // A2B: binary sharings of both parties' shares (ZERO_BIN masks).
  const Quad4 m = quad_gen(seed, op_mask, stream_word2(MPC_ROLE_ZERO_BIN, 0, 0), op_mask,
                           stream_word2(MPC_ROLE_ZERO_BIN, 0, 1), op_mask,
                           stream_word2(MPC_ROLE_ZERO_BIN, 1, 0), op_mask,
                           stream_word2(MPC_ROLE_ZERO_BIN, 1, 1), blk, j);
  const Sh2 u{{m.w[0] ^ m.w[1] ^ y.v[0], m.w[1] ^ m.w[0]}};
  const Sh2 v{{m.w[2] ^ m.w[3], m.w[3] ^ m.w[2] ^ y.v[1]}};
  // Kogge-Stone: gate g uses AND_A/B (g, 0/1) and AND_C (g, 0).
  Quad4 c0s[3];
#pragma unroll
  for (int q = 0; q < 3; ++q)
    c0s[q] = quad_gen(seed, op_and, stream_word2(MPC_ROLE_AND_C, 4 * q + 0, 0), op_and,
                      stream_word2(MPC_ROLE_AND_C, 4 * q + 1, 0), op_and,
                      stream_word2(MPC_ROLE_AND_C, 4 * q + 2, 0), op_and,
                      stream_word2(MPC_ROLE_AND_C, 4 * q + 3, 0), blk, j);
  auto gate_ab = [&](int g) {
    return quad_gen(seed, op_and, stream_word2(MPC_ROLE_AND_A, g, 0), op_and,
                    stream_word2(MPC_ROLE_AND_A, g, 1), op_and,
                    stream_word2(MPC_ROLE_AND_B, g, 0), op_and,
                    stream_word2(MPC_ROLE_AND_B, g, 1), blk, j);
  };
  int gate = 0;
  Sh2 G = and2(u, v, gate_ab(gate), c0s[0].w[0]);
  ++gate;
  Sh2 Pp = xr2(u, v);
  const Sh2 P0 = Pp;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int d = 1 << r;
    const Sh2 t = and2(Pp, shl2(G, d), gate_ab(gate), c0s[gate >> 2].w[gate & 3]);
    ++gate;
    if (d < 32) {
      Pp = and2(Pp, shl2(Pp, d), gate_ab(gate), c0s[gate >> 2].w[gate & 3]);
      ++gate;
    }
    G = xr2(G, t);
  }
  const Sh2 sb = xr2(P0, shl2(G, 1));
  // B2A pair (r, <r>_0, [r]_0) plus the spare stream.
  const Quad4 rq = quad_gen(seed, op_b2a, stream_word2(MPC_ROLE_B2A_R, 0, MPC_TTP_PARTY), op_b2a,
                            stream_word2(MPC_ROLE_B2A_BIN, 0, 0), op_b2a,
                            stream_word2(MPC_ROLE_B2A_ARITH, 0, 0), extra_op, extra_w2, blk, j);
  extra = rq.w[3];
  const u64 rbit = rq.w[0] & 1ull;  // <r>_0 ^ <r>_1 = r
  const u64 z = ((sb.v[0] ^ sb.v[1]) >> 63) ^ rbit;
  const u64 ra0 = rq.w[2], ra1 = rbit - rq.w[2];
  return Sh2{{ra0 - 2ull * z * ra0 + z, ra1 - 2ull * z * ra1}};
}

// ---- arithmetic steps (two parties) --------------------------------------------------
__device__ __forceinline__ Sh2 trunc2(Sh2 z, int bits) {
  return bits ? Sh2{{sar(z.v[0], bits), sar(z.v[1], bits)}} : z;
}

// Beaver product (App. D.1.1) with triple words a_0, a_1, b_0, b_1, c_0 and
// c_1 = (a_0 + a_1)(b_0 + b_1) - c_0; party 0 adds eps * delta.  Then truncation.
__device__ __forceinline__ Sh2 mul2(Sh2 x, Sh2 y, const u64* w, int trunc_bits) {
  const u64 A0 = w[0], A1 = w[1], B0 = w[2], B1 = w[3], C0 = w[4];
  const u64 C1 = (A0 + A1) * (B0 + B1) - C0;
  const u64 E = (x.v[0] - A0) + (x.v[1] - A1);
  const u64 F = (y.v[0] - B0) + (y.v[1] - B1);
  return trunc2(Sh2{{C0 + E * B0 + A0 * F + E * F, C1 + E * B1 + A1 * F}}, trunc_bits);
}

// Beaver square with the pair words a_0, a_1, b_0 and b_1 = (a_0 + a_1)^2 - b_0:
// [x^2] = [b] + 2 eps [a] + eps^2 (party 0).  Then truncation.
__device__ __forceinline__ Sh2 sq2(Sh2 x, const u64* w, int trunc_bits) {
  const u64 A0 = w[0], A1 = w[1], B0 = w[2];
  const u64 a = A0 + A1;
  const u64 B1 = a * a - B0;
  const u64 E = (x.v[0] - A0) + (x.v[1] - A1);
  return trunc2(Sh2{{B0 + 2ull * E * A0 + E * E, B1 + 2ull * E * A1}}, trunc_bits);
}

// Public affine map per share: scale * x_p (+ offset on party 0), then truncation.
__device__ __forceinline__ Sh2 affine2(Sh2 x, u64 scale, u64 offset, int trunc_bits = 0) {
  return trunc2(Sh2{{x.v[0] * scale + offset, x.v[1] * scale}}, trunc_bits);
}

__device__ __forceinline__ Sh2 add2(Sh2 a, Sh2 b) { return Sh2{{a.v[0] + b.v[0], a.v[1] + b.v[1]}}; }
__device__ __forceinline__ Sh2 sub2(Sh2 a, Sh2 b) { return Sh2{{a.v[0] - b.v[0], a.v[1] - b.v[1]}}; }

// ReLU([x]) = [x] * [x > 0] (Section 5.2): [x > 0] = [-x < 0] from ltz_quad with
// material at op, op + 1, op + 3, then the Beaver product with the elementwise
// triple at op + 2 (no truncation: [x > 0] is an unscaled 0/1 sharing).  The
// triple's c_0 rides in the B2A group's spare slot.
__device__ __forceinline__ Sh2 relu_quad(Sh2 x, u64 seed, u64 op, i64 blk, int j) {
  const u64 op_mul = op + 2;
  u64 w[5];
  const Sh2 bit = ltz_quad(Sh2{{0ull - x.v[0], 0ull - x.v[1]}}, seed, op, blk, j, op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_C, 0, 0), w[4]);
  const Quad4 t = quad_gen(seed, op_mul, stream_word2(MPC_ROLE_TRIPLE_A, 0, 0), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_A, 0, 1), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_B, 0, 0), op_mul,
                           stream_word2(MPC_ROLE_TRIPLE_B, 0, 1), blk, j);
#pragma unroll
  for (int s = 0; s < 4; ++s) w[s] = t.w[s];
  return mul2(x, bit, w, 0);
}

// ---- word lists: the streams of consecutive steps, generated four at a time ----------
// A step at op id `op` reads, for this element, the words of
//   square: TRIPLE_A (p = 0, 1), TRIPLE_C (p = 0)                       -- 3 words
//   product: TRIPLE_A (p = 0, 1), TRIPLE_B (p = 0, 1), TRIPLE_C (p = 0)  -- 5 words
// A chunk lists the words of several steps in order (padded to a multiple of
// four with repeats of the first stream) and generates them with N/4 quad_gen.
template <int N>
struct WordList {
  u64 op[N], w2[N], w[N];
  int len = 0;
  __device__ __forceinline__ void add(u64 o, u64 word2) {
    op[len] = o;
    w2[len] = word2;
    ++len;
  }
  __device__ __forceinline__ void add_square(u64 o) {
    add(o, stream_word2(MPC_ROLE_TRIPLE_A, 0, 0));
    add(o, stream_word2(MPC_ROLE_TRIPLE_A, 0, 1));
    add(o, stream_word2(MPC_ROLE_TRIPLE_C, 0, 0));
  }
  __device__ __forceinline__ void add_mul(u64 o) {
    add(o, stream_word2(MPC_ROLE_TRIPLE_A, 0, 0));
    add(o, stream_word2(MPC_ROLE_TRIPLE_A, 0, 1));
    add(o, stream_word2(MPC_ROLE_TRIPLE_B, 0, 0));
    add(o, stream_word2(MPC_ROLE_TRIPLE_B, 0, 1));
    add(o, stream_word2(MPC_ROLE_TRIPLE_C, 0, 0));
  }
  __device__ __forceinline__ void generate(u64 seed, i64 blk, int j) {
    static_assert(N % 4 == 0, "word lists hold whole groups");
    const u64 pad_op = op[0], pad_w2 = w2[0];
#pragma unroll
    for (int k = 0; k < N; ++k)  // fixed trip count: folds to straight-line code
      if (k >= len) {
        op[k] = pad_op;
        w2[k] = pad_w2;
      }
#pragma unroll
    for (int g = 0; g < N / 4; ++g) {
      const Quad4 q = quad_gen(seed, op[4 * g], w2[4 * g], op[4 * g + 1], w2[4 * g + 1],
                               op[4 * g + 2], w2[4 * g + 2], op[4 * g + 3], w2[4 * g + 3], blk, j);
#pragma unroll
      for (int s = 0; s < 4; ++s) w[4 * g + s] = q.w[s];
    }
  }
};

}  // namespace mpc
