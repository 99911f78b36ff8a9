// Truncation for any number of parties with the wrap count of Alg. 1.
//
// With signed views s(.) of ring elements, x = sum_p s(x_p) - theta_x Q.  The
// dealer supplies a uniform [r] and shares of its wrap count theta_r; the
// parties open z = x + r (one round), and
//     [theta_x] = theta_z + [beta] - [theta_r]     (eta set to 0, as the paper does)
// with beta_p the signed overflow of the local addition x_p + r_p and theta_z
// the wrap count of the opened shares.  Each party then keeps
//     floor(s(x_p) / 2^f) - [theta_x]_p 2^(64 - f).
// Setting eta to 0 is wrong when the signed plaintext sum x + r overflows,
// which happens with probability about |x| / 2^64.
#include "common.cuh"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ i64 sv(u64 v) { return (i64)v; }

// Wrap count of a signed 128-bit sum S of P signed words: (S - s(S mod Q)) / Q.
__device__ __forceinline__ i64 wraps_of(__int128 S) {
  const i64 low = (i64)(u64)S;
  return (i64)((S - (__int128)low) >> 64);
}

__global__ void __launch_bounds__(kThreads) trunc_pairs_kernel(int P, i64 n, u64 seed, u64 op_id,
                                                               u64* __restrict__ R,
                                                               u64* __restrict__ TH) {
  const i64 nblk = ceil_div(n, 4);
  for (i64 t = blockIdx.x * (i64)blockDim.x + threadIdx.x; t < nblk;
       t += (i64)gridDim.x * blockDim.x) {
    const i64 i0 = 4 * t;
    __int128 S[4] = {0, 0, 0, 0};
    for (int p = 0; p < P; ++p) {
      const u64x4 r = prg_block(seed, op_id, stream_word2(MPC_ROLE_TRUNC_R, 0, p), t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) R[(i64)p * n + i0 + j] = r.v[j];
        S[j] += (__int128)sv(r.v[j]);
      }
    }
    u64 acc[4] = {0, 0, 0, 0};
    for (int p = 0; p < P - 1; ++p) {
      const u64x4 h = prg_block(seed, op_id, stream_word2(MPC_ROLE_TRUNC_R, 1, p), t);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (i0 + j < n) TH[(i64)p * n + i0 + j] = h.v[j];
        acc[j] += h.v[j];
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (i0 + j < n) TH[(i64)(P - 1) * n + i0 + j] = (u64)wraps_of(S[j]) - acc[j];
  }
}

template <int P>
__global__ void __launch_bounds__(kThreads) trunc_nparty_kernel(i64 n, u64* X,
                                                                const u64* __restrict__ R,
                                                                const u64* __restrict__ TH,
                                                                int f) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    u64 x[P], z[P];
    i64 beta[P];
    __int128 Sz = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      x[p] = X[(i64)p * n + i];
      const u64 r = R[(i64)p * n + i];
      z[p] = x[p] + r;
      beta[p] = wraps_of((__int128)sv(x[p]) + (__int128)sv(r));  // s(x_p)+s(r_p) = s(z_p)+beta_p Q
      Sz += (__int128)sv(z[p]);
    }
    const i64 theta_z = wraps_of(Sz);  // from the opened z
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const u64 th = (u64)beta[p] - TH[(i64)p * n + i] + (p == 0 ? (u64)theta_z : 0ull);
      X[(i64)p * n + i] = (u64)(sv(x[p]) >> f) - (th << (64 - f));
    }
  }
}

template <int P>
void launch_nparty(i64 n, u64* X, const u64* R, const u64* TH, int f, cudaStream_t s) {
  trunc_nparty_kernel<P><<<grid_for(n, kThreads), kThreads, 0, s>>>(n, X, R, TH, f);
}

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" {

int mpc_ttp_trunc_pairs(int P, int64_t n, uint64_t seed, uint64_t op_id, uint64_t* r,
                        uint64_t* theta_r, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(r && theta_r, "null pointer");
  trunc_pairs_kernel<<<grid_for(ceil_div(n, 4), kThreads), kThreads, 0, as_stream(stream)>>>(
      P, n, seed, op_id, (u64*)r, (u64*)theta_r);
  return check_launch("ttp_trunc_pairs");
}

int mpc_truncate_nparty(int P, int64_t n, uint64_t* shares, const uint64_t* r,
                        const uint64_t* theta_r, int frac_bits, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(n >= 0, "negative length");
  MPC_REQUIRE(frac_bits >= 1 && frac_bits <= 63, "frac_bits %d outside [1, 63]", frac_bits);
  if (n == 0) return MPC_OK;
  MPC_REQUIRE(shares && r && theta_r, "null pointer");
  MPC_DISPATCH_P(P, launch_nparty, n, (u64*)shares, (const u64*)r, (const u64*)theta_r,
                 frac_bits, as_stream(stream));
  int rc = check_launch("truncate_nparty");
  if (rc == MPC_OK) stats_add(1, 8ull * (uint64_t)n, 0, 2ull * P * (uint64_t)n, 0);
  return rc;
}

}  // extern "C"
