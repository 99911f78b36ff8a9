// Binary shares for two parties: A2B with a Kogge-Stone adder, and the fused
// private ReLU = Beaver(x, B2A(MSB(A2B(-x)))) (§5.2 "Comparators", App.
// D.1.2-D.1.4, Alg. 2).  One kernel, one pass: every opening (the 12 AND
// gates' eps/delta, the B2A bit z, the Beaver E/F) is an XOR/sum of the two
// parties' registers.  Each thread owns 4 consecutive elements, i.e. one
// Philox block of each binary zero-share stream.
#include "common.cuh"
#include "host.hpp"

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
__device__ __forceinline__ Pair a2b_block(const Pair& y, const u64* __restrict__ T, i64 n, i64 i0,
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
  Pair G = and_gate(u, v, T, gate++, n, i0);
  Pair Pp = xr(u, v);
  const Pair P0 = Pp;
#pragma unroll
  for (int r = 0; r < 6; ++r) {
    const int d = 1 << r;  // 1, 2, 4, 8, 16, 32
    const Pair Gn = xr(G, and_gate(Pp, shl(G, d), T, gate++, n, i0));
    if (d < 32) Pp = and_gate(Pp, shl(Pp, d), T, gate++, n, i0);
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
    const Pair b = a2b_block(x, T, n, i0, t, seed, op_id);
    store4(Bout, i0, n, b.s[0]);
    store4(Bout + n, i0, n, b.s[1]);
  }
}

__global__ void __launch_bounds__(kThreads) relu_kernel(i64 n, const u64* X, u64* Y,
                                                        const u64* __restrict__ T,
                                                        const u64* __restrict__ r_arith,
                                                        const u64* __restrict__ r_bin,
                                                        const u64* __restrict__ MT, u64 seed,
                                                        u64 op_id) {
  const i64 nblk = ceil_div(n, 4);
  const i64 nw = ceil_div(n, 64);
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
    const Pair sb = a2b_block(neg, T, n, i0, t, seed, op_id);
    // B2A (Alg. 2): z = reveal(<b> ^ <r>), [b]_p = [r]_p - 2 z [r]_p + [p = 0] z.
    const int sh = (int)(i0 & 63);
    const u64 rb0 = r_bin[i0 >> 6] >> sh, rb1 = r_bin[nw + (i0 >> 6)] >> sh;
    const Quad ra0 = load4(r_arith, i0, n), ra1 = load4(r_arith + n, i0, n);
    Pair bit;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const u64 z = ((sb.s[0].v[j] ^ sb.s[1].v[j]) >> 63) ^ ((rb0 ^ rb1) >> j & 1ull);
      bit.s[0].v[j] = ra0.v[j] - 2ull * z * ra0.v[j] + z;
      bit.s[1].v[j] = ra1.v[j] - 2ull * z * ra1.v[j];
    }
    // Beaver product x * [b] (no truncation: the mask is an unscaled 0/1).
    const Quad A0 = load4(MT, i0, n), A1 = load4(MT + n, i0, n);
    const Quad B0 = load4(MT + 2 * n, i0, n), B1 = load4(MT + 3 * n, i0, n);
    const Quad C0 = load4(MT + 4 * n, i0, n), C1 = load4(MT + 5 * n, i0, n);
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

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_a2b(int P, int64_t n, const uint64_t* arith, uint64_t* binary,
            const uint64_t* and_triples, uint64_t seed, uint64_t op_id, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "A2B supports P = 2 only (got %d)", P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(arith && binary && and_triples, "null pointer");
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
                     const uint64_t* r_bin, const uint64_t* mul_triple, uint64_t seed,
                     uint64_t op_id, void* stream) {
  if (P != 2) return fail(P >= 1 && P <= MPC_MAX_PARTIES ? MPC_EUNSUPPORTED : MPC_EINVAL,
                          "private ReLU supports P = 2 only (got %d)", P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y && and_triples && r_arith && r_bin && mul_triple, "null pointer");
  int rc;
  {
    KernelTimer timer("private_relu", as_stream(stream));
    relu_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
        n, (const u64*)X, (u64*)Y, (const u64*)and_triples, (const u64*)r_arith,
        (const u64*)r_bin, (const u64*)mul_triple, seed, op_id);
    rc = check_launch("private_relu");
  }
  if (rc == MPC_OK)
    stats_add(9, (uint64_t)MPC_KS_GATES * 16ull * n + (uint64_t)ceil_div(n, 8) + 16ull * n,
              (uint64_t)MPC_KS_GATES * n, (uint64_t)MPC_KS_GATES * 6ull * n + 2ull * n + 6ull * n,
              0);
  return rc;
}

}  // extern "C"
