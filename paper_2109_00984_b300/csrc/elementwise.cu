// HBM-bound elementwise kernels: sharing, reveal, dealer fills, fused Beaver
// product, truncation.  Each thread owns one Philox block = 4 consecutive words.
#include <math.h>

#include "common.cuh"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int kThreads = 256;

// ---- sharing (§5.1) -------------------------------------------------------------
// shares[p] = R_p - R_{(p-1) mod P} + [p == src] x, R_p = stream(ZERO_ARITH, 0, p).
template <bool kEncode>
__global__ void __launch_bounds__(kThreads) share_kernel(const double* __restrict__ xr,
                                                         const u64* __restrict__ xe, i64 n,
                                                         int P, int src, int frac_bits,
                                                         u64 seed, u64 op_id,
                                                         u64* __restrict__ shares,
                                                         int* status) {
  const i64 nblk = ceil_div(n, 4);
  const double scale = ldexp(1.0, frac_bits);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad x;
    if (kEncode) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        u64 v = 0;
        if (i0 + j < n) {
          const double s = xr[i0 + j] * scale;
          if (isfinite(s) && fabs(s) < 9223372036854775808.0) {
            v = (u64)__double2ll_rn(s);
          } else {
            record_status(status, MPC_ERANGE);
          }
        }
        x.v[j] = v;
      }
    } else {
      x = load4(xe, i0, n);
    }
    const u64x4 last = prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_ARITH, 0, P - 1), t);
    u64x4 prev = last;
    for (int p = 0; p < P; ++p) {
      const u64x4 cur =
          (p == P - 1) ? last : prg_block(seed, op_id, stream_word2(MPC_ROLE_ZERO_ARITH, 0, p), t);
      Quad s;
#pragma unroll
      for (int j = 0; j < 4; ++j) s.v[j] = cur.v[j] - prev.v[j] + (p == src ? x.v[j] : 0ull);
      store4(shares + (i64)p * n, i0, n, s);
      prev = cur;
    }
  }
}

// ---- reveal --------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) reveal_kernel(const u64* __restrict__ shares, int P,
                                                          i64 n, int frac_bits,
                                                          u64* __restrict__ ring_out,
                                                          double* __restrict__ real_out) {
  const i64 nblk = ceil_div(n, 4);
  const double inv = ldexp(1.0, -frac_bits);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad acc = load4(shares, i0, n);
    for (int p = 1; p < P; ++p) {
      const Quad s = load4(shares + (i64)p * n, i0, n);
#pragma unroll
      for (int j = 0; j < 4; ++j) acc.v[j] += s.v[j];
    }
    if (ring_out) store4(ring_out, i0, n, acc);
    if (real_out) {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (i0 + j < n) real_out[i0 + j] = (double)(i64)acc.v[j] * inv;
    }
  }
}

// ---- dealer: elementwise Beaver triples ---------------------------------------------
__global__ void __launch_bounds__(kThreads) mul_triple_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                              u64* __restrict__ A,
                                                              u64* __restrict__ B,
                                                              u64* __restrict__ C) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad a = {{0, 0, 0, 0}}, b = {{0, 0, 0, 0}}, cs = {{0, 0, 0, 0}};
    for (int p = 0; p < P; ++p) {
      const Quad ap = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_A, 0, p), t));
      const Quad bp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_B, 0, p), t));
      store4(A + (i64)p * n, i0, n, ap);
      store4(B + (i64)p * n, i0, n, bp);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a.v[j] += ap.v[j];
        b.v[j] += bp.v[j];
      }
    }
    for (int p = 0; p < P - 1; ++p) {
      const Quad cp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_C, 0, p), t));
      store4(C + (i64)p * n, i0, n, cp);
#pragma unroll
      for (int j = 0; j < 4; ++j) cs.v[j] += cp.v[j];
    }
    Quad last;
#pragma unroll
    for (int j = 0; j < 4; ++j) last.v[j] = a.v[j] * b.v[j] - cs.v[j];
    store4(C + (i64)(P - 1) * n, i0, n, last);
  }
}

// ---- dealer: binary AND triples --------------------------------------------------------
// T layout [gates][3][P][n]; grid.y = gate.
__global__ void __launch_bounds__(kThreads) and_triples_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                               u64* __restrict__ T) {
  const int g = blockIdx.y;
  const i64 nblk = ceil_div(n, 4);
  u64* Ta = T + ((i64)g * 3 + 0) * P * n;
  u64* Tb = T + ((i64)g * 3 + 1) * P * n;
  u64* Tc = T + ((i64)g * 3 + 2) * P * n;
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad a = {{0, 0, 0, 0}}, b = {{0, 0, 0, 0}}, cs = {{0, 0, 0, 0}};
    for (int p = 0; p < P; ++p) {
      const Quad ap = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_AND_A, g, p), t));
      const Quad bp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_AND_B, g, p), t));
      store4(Ta + (i64)p * n, i0, n, ap);
      store4(Tb + (i64)p * n, i0, n, bp);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a.v[j] ^= ap.v[j];
        b.v[j] ^= bp.v[j];
      }
    }
    for (int p = 0; p < P - 1; ++p) {
      const Quad cp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_AND_C, g, p), t));
      store4(Tc + (i64)p * n, i0, n, cp);
#pragma unroll
      for (int j = 0; j < 4; ++j) cs.v[j] ^= cp.v[j];
    }
    Quad last;
#pragma unroll
    for (int j = 0; j < 4; ++j) last.v[j] = (a.v[j] & b.v[j]) ^ cs.v[j];
    store4(Tc + (i64)(P - 1) * n, i0, n, last);
  }
}

// ---- dealer: B2A random-bit pairs ---------------------------------------------------
// Arithmetic half: [r]_p for p < P-1 from B2A_ARITH, last = r - sum.
__global__ void __launch_bounds__(kThreads) b2a_arith_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                             u64* __restrict__ r_arith) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    const u64x4 r = prg_block(seed, op_id, stream_word2(MPC_ROLE_B2A_R, 0, MPC_TTP_PARTY), t);
    Quad acc = {{0, 0, 0, 0}};
    for (int p = 0; p < P - 1; ++p) {
      const Quad rp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_B2A_ARITH, 0, p), t));
      store4(r_arith + (i64)p * n, i0, n, rp);
#pragma unroll
      for (int j = 0; j < 4; ++j) acc.v[j] += rp.v[j];
    }
    Quad last;
#pragma unroll
    for (int j = 0; j < 4; ++j) last.v[j] = (r.v[j] & 1ull) - acc.v[j];
    store4(r_arith + (i64)(P - 1) * n, i0, n, last);
  }
}

// Binary half, bit-packed: one thread per 64-element word.
__global__ void __launch_bounds__(kThreads) b2a_bin_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                           u64* __restrict__ r_bin) {
  const i64 nw = ceil_div(n, 64);
  for (i64 w = blockIdx.x * (i64)blockDim.x + threadIdx.x; w < nw;
       w += (i64)gridDim.x * blockDim.x) {
    const int valid = (int)min((i64)64, n - 64 * w);
    const u64 mask = valid == 64 ? ~0ull : ((1ull << valid) - 1ull);
    u64 rw = 0;
    for (int b = 0; b < 16; ++b) {
      const u64x4 r = prg_block(seed, op_id, stream_word2(MPC_ROLE_B2A_R, 0, MPC_TTP_PARTY),
                                16 * w + b);
#pragma unroll
      for (int j = 0; j < 4; ++j) rw |= (r.v[j] & 1ull) << (4 * b + j);
    }
    u64 acc = 0;
    for (int p = 0; p < P - 1; ++p) {
      u64 word = 0;
      for (int b = 0; b < 16; ++b) {
        const u64x4 r = prg_block(seed, op_id, stream_word2(MPC_ROLE_B2A_BIN, 0, p), 16 * w + b);
#pragma unroll
        for (int j = 0; j < 4; ++j) word |= (r.v[j] & 1ull) << (4 * b + j);
      }
      word &= mask;
      r_bin[(i64)p * nw + w] = word;
      acc ^= word;
    }
    r_bin[(i64)(P - 1) * nw + w] = (rw & mask) ^ acc;
  }
}

// ---- fused Beaver elementwise product (App. D.1.1) ---------------------------------------
// One pass: open E, F in registers, combine, optionally truncate.
template <int P>
__global__ void __launch_bounds__(kThreads) beaver_mul_kernel(
    i64 n, const u64* X, const u64* Y, const u64* __restrict__ A,
    const u64* __restrict__ B, const u64* __restrict__ C, u64* Z, u64* __restrict__ E_out,
    u64* __restrict__ F_out, int trunc_bits) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad a[P], b[P];
    Quad e = {{0, 0, 0, 0}}, f = {{0, 0, 0, 0}};
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const Quad x = load4(X + (i64)p * n, i0, n);
      const Quad y = load4(Y + (i64)p * n, i0, n);
      a[p] = load4(A + (i64)p * n, i0, n);
      b[p] = load4(B + (i64)p * n, i0, n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        e.v[j] += x.v[j] - a[p].v[j];
        f.v[j] += y.v[j] - b[p].v[j];
      }
    }
    if (E_out) store4(E_out, i0, n, e);
    if (F_out) store4(F_out, i0, n, f);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Quad z = load4(C + (i64)p * n, i0, n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        z.v[j] += e.v[j] * b[p].v[j] + a[p].v[j] * f.v[j];
        if (p == 0) z.v[j] += e.v[j] * f.v[j];
        if (trunc_bits > 0) z.v[j] = sar(z.v[j], trunc_bits);
      }
      store4(Z + (i64)p * n, i0, n, z);
    }
  }
}

template <int P>
void launch_beaver_mul(i64 n, const u64* X, const u64* Y, const u64* A, const u64* B,
                       const u64* C, u64* Z, u64* E, u64* F, int trunc_bits, cudaStream_t s) {
  KernelTimer timer("beaver_mul", s);
  beaver_mul_kernel<P><<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, s>>>(
      n, X, Y, A, B, C, Z, E, F, trunc_bits);
}

// ---- two-party local truncation ------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) truncate_kernel(i64 total, u64* __restrict__ s,
                                                            int frac_bits, i64 divisor) {
  const i64 nblk = ceil_div(total, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad q = load4(s, i0, total);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      q.v[j] = divisor > 0 ? floordiv_signed(q.v[j], divisor) : sar(q.v[j], frac_bits);
    store4(s, i0, total, q);
  }
}

// ---- Beaver square (App. D.1.1 "Square") and the public affine map --------------------
// Dealer pair: A[p] = TRIPLE_A(p), b = a^2 shared with TRIPLE_C words + correction.
__global__ void __launch_bounds__(kThreads) square_pair_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                               u64* __restrict__ A,
                                                               u64* __restrict__ B) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad a = {{0, 0, 0, 0}}, cs = {{0, 0, 0, 0}};
    for (int p = 0; p < P; ++p) {
      const Quad ap = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_A, 0, p), t));
      store4(A + (i64)p * n, i0, n, ap);
#pragma unroll
      for (int j = 0; j < 4; ++j) a.v[j] += ap.v[j];
    }
    for (int p = 0; p < P - 1; ++p) {
      const Quad bp = as_quad(prg_block(seed, op_id, stream_word2(MPC_ROLE_TRIPLE_C, 0, p), t));
      store4(B + (i64)p * n, i0, n, bp);
#pragma unroll
      for (int j = 0; j < 4; ++j) cs.v[j] += bp.v[j];
    }
    Quad last;
#pragma unroll
    for (int j = 0; j < 4; ++j) last.v[j] = a.v[j] * a.v[j] - cs.v[j];
    store4(B + (i64)(P - 1) * n, i0, n, last);
  }
}

// Z_p = B_p + 2 eps A_p (+ eps^2 on party 0), eps = sum_p (X_p - A_p) opened in registers.
template <int P>
__global__ void __launch_bounds__(kThreads) beaver_square_kernel(i64 n, const u64* X,
                                                                 const u64* __restrict__ A,
                                                                 const u64* __restrict__ B,
                                                                 u64* Z, int trunc_bits) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    Quad a[P];
    Quad e = {{0, 0, 0, 0}};
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const Quad x = load4(X + (i64)p * n, i0, n);
      a[p] = load4(A + (i64)p * n, i0, n);
#pragma unroll
      for (int j = 0; j < 4; ++j) e.v[j] += x.v[j] - a[p].v[j];
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Quad z = load4(B + (i64)p * n, i0, n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        z.v[j] += 2ull * e.v[j] * a[p].v[j];
        if (p == 0) z.v[j] += e.v[j] * e.v[j];
        if (trunc_bits > 0) z.v[j] = sar(z.v[j], trunc_bits);
      }
      store4(Z + (i64)p * n, i0, n, z);
    }
  }
}

template <int P>
void launch_beaver_square(i64 n, const u64* X, const u64* A, const u64* B, u64* Z, int trunc_bits,
                          cudaStream_t s) {
  beaver_square_kernel<P><<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, s>>>(n, X, A, B, Z,
                                                                                 trunc_bits);
}

// Z_p = scale X_p (+ offset on party 0), then optionally s(Z_p) >> trunc_bits.
__global__ void __launch_bounds__(kThreads) affine_kernel(int P, i64 n, const u64* X, u64* Z,
                                                          u64 scale, u64 offset, int trunc_bits) {
  const i64 total = (i64)P * n;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    u64 v = X[i] * scale + (i < n ? offset : 0ull);
    if (trunc_bits > 0) v = sar(v, trunc_bits);
    Z[i] = v;
  }
}

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_ring_share(const double* x, int64_t n, int P, int src, int frac_bits, uint64_t seed,
                   uint64_t op_id, uint64_t* shares, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(src >= 0 && src < P, "source party %d outside [0, %d)", src, P);
  MPC_REQUIRE(frac_bits >= 0 && frac_bits <= 62, "frac_bits %d outside [0, 62]", frac_bits);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(x != nullptr && shares != nullptr, "null pointer");
  int* st = device_status_ptr();
  if (!st) return fail(MPC_ECUDA, "device status word unavailable");
  share_kernel<true><<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      x, nullptr, n, P, src, frac_bits, seed, op_id, (u64*)shares, st);
  return check_launch("ring_share");
}

int mpc_ring_share_encoded(const uint64_t* x_ring, int64_t n, int P, int src, uint64_t seed,
                           uint64_t op_id, uint64_t* shares, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(src >= 0 && src < P, "source party %d outside [0, %d)", src, P);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(x_ring != nullptr && shares != nullptr, "null pointer");
  share_kernel<false><<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      nullptr, (const u64*)x_ring, n, P, src, 0, seed, op_id, (u64*)shares, nullptr);
  return check_launch("ring_share_encoded");
}

int mpc_reveal(const uint64_t* shares, int P, int64_t n, int frac_bits, uint64_t* ring_out,
               double* real_out, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(frac_bits >= 0 && frac_bits <= 63, "frac_bits %d outside [0, 63]", frac_bits);
  MPC_REQUIRE(ring_out != nullptr || real_out != nullptr, "both outputs are null");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(shares != nullptr, "null shares");
  reveal_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      (const u64*)shares, P, n, frac_bits, (u64*)ring_out, real_out);
  return check_launch("reveal");
}

int mpc_ttp_mul_triple(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* A, uint64_t* B,
                       uint64_t* C, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(A && B && C, "null pointer");
  mul_triple_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      P, n, seed, op_id, (u64*)A, (u64*)B, (u64*)C);
  return check_launch("ttp_mul_triple");
}

int mpc_ttp_and_triples(int P, int64_t n, int gates, uint64_t seed, uint64_t op_id, uint64_t* T,
                        void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(gates >= 1 && gates <= 65535, "gate count %d outside [1, 65535]", gates);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(T != nullptr, "null pointer");
  dim3 grid(grid_for(ceil_div(n, 4), kThreads, 148 * 8), gates);
  and_triples_kernel<<<grid, kThreads, 0, as_stream(stream)>>>(P, n, seed, op_id, (u64*)T);
  return check_launch("ttp_and_triples");
}

int mpc_ttp_b2a_bits(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* r_arith,
                     uint64_t* r_bin, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(r_arith && r_bin, "null pointer");
  cudaStream_t s = as_stream(stream);
  b2a_arith_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, s>>>(P, n, seed, op_id,
                                                                           (u64*)r_arith);
  int rc = check_launch("ttp_b2a_bits/arith");
  if (rc) return rc;
  b2a_bin_kernel<<<grid_for(ceil_div(n, 64), 128), 128, 0, s>>>(P, n, seed, op_id, (u64*)r_bin);
  return check_launch("ttp_b2a_bits/bin");
}

int mpc_beaver_mul(int P, int64_t n, const uint64_t* X, const uint64_t* Y, const uint64_t* A,
                   const uint64_t* B, const uint64_t* C, uint64_t* Z, uint64_t* E_out,
                   uint64_t* F_out, int trunc_bits, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Y && A && B && C && Z, "null pointer");
  MPC_DISPATCH_P(P, launch_beaver_mul, n, (const u64*)X, (const u64*)Y, (const u64*)A,
                 (const u64*)B, (const u64*)C, (u64*)Z, (u64*)E_out, (u64*)F_out, trunc_bits,
                 as_stream(stream));
  int rc = check_launch("beaver_mul");
  if (rc == MPC_OK) stats_add(1, 2ull * 8ull * (uint64_t)n, 0, 3ull * P * (uint64_t)n, 0);
  return rc;
}

int mpc_truncate(int P, int64_t n, uint64_t* shares, int frac_bits, int64_t divisor,
                 void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(frac_bits >= 0 && frac_bits <= 63, "frac_bits %d outside [0, 63]", frac_bits);
  MPC_REQUIRE(divisor >= 0, "negative divisor");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(shares != nullptr, "null pointer");
  const i64 total = (i64)P * n;
  truncate_kernel<<<grid_for(ceil_div(total, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      total, (u64*)shares, frac_bits, divisor);
  int rc = check_launch("truncate");
  if (rc == MPC_OK) stats_add(0, 0, 0, 0, 0);
  return rc;
}

int mpc_ttp_square_pair(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* A, uint64_t* B,
                        void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(A && B, "null pointer");
  square_pair_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      P, n, seed, op_id, (u64*)A, (u64*)B);
  return check_launch("ttp_square_pair");
}

int mpc_beaver_square(int P, int64_t n, const uint64_t* X, const uint64_t* A, const uint64_t* B,
                      uint64_t* Z, int trunc_bits, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && A && B && Z, "null pointer");
  MPC_DISPATCH_P(P, launch_beaver_square, n, (const u64*)X, (const u64*)A, (const u64*)B, (u64*)Z,
                 trunc_bits, as_stream(stream));
  int rc = check_launch("beaver_square");
  if (rc == MPC_OK) stats_add(1, 8ull * (uint64_t)n, 0, 2ull * P * (uint64_t)n, 0);
  return rc;
}

int mpc_affine(int P, int64_t n, const uint64_t* X, uint64_t* Z, int64_t scale, uint64_t offset,
               int trunc_bits, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(X && Z, "null pointer");
  affine_kernel<<<grid_for((i64)P * n, kThreads), kThreads, 0, as_stream(stream)>>>(
      P, n, (const u64*)X, (u64*)Z, (u64)scale, (u64)offset, trunc_bits);
  return check_launch("affine");
}

}  // extern "C"
