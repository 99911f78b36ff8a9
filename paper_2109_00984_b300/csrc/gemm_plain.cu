// Plain ring GEMM on CUDA cores: 64-bit multiply-add modulo 2^64 emulated by
// the compiler on 32-bit integer multiply-add units.  This is the baseline the
// tensor-core limb engine is measured against.
//
// Tile 128x128 per CTA, K step 8, 256 threads with an 8x8 register tile each;
// operands staged through shared memory with a register-prefetched double
// buffer.  Rows/columns of a thread are interleaved in pairs so that every
// 16-byte shared-memory read of a quarter-warp is contiguous.
#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

namespace {

constexpr int BM = 128, BN = 128, BK = 8, kThreads = 256;
constexpr int APAD = 2;  // keeps rows 16-byte aligned and staggers banks

__device__ __forceinline__ int frag_idx(int i, int t) { return 32 * (i >> 1) + 2 * t + (i & 1); }

__global__ void __launch_bounds__(kThreads, 1) gemm_plain_kernel(const GemmArgs g) {
  __shared__ __align__(16) u64 As[2][BK][BM + APAD];
  __shared__ __align__(16) u64 Bs[2][BK][BN];

  const GemmJob& job = g.jobs[blockIdx.z];
  const i64 M = g.M, N = g.N, K = g.K;
  const i64 m0 = (i64)blockIdx.y * BM, n0 = (i64)blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int npairs = job.A2 ? 2 : 1;
  const i64 ktiles = ceil_div(K, BK);
  const i64 total_tiles = ktiles * npairs;

  // Global-load coordinates.
  const int a_r = tid >> 1, a_k = (tid & 1) * 4;   // A: row a_r, 4 consecutive k
  const int b_k = tid >> 5, b_n = (tid & 31) * 4;  // B: k row b_k, 4 consecutive n

  u64 ra[4], rb[4];
  auto fetch = [&](i64 kt) {
    const int pair = (int)(kt / ktiles);
    const i64 k0 = (kt % ktiles) * BK;
    const u64* A = pair ? job.A2 : job.A1;
    const u64* B = pair ? job.B2 : job.B1;
    const i64 row = m0 + a_r;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const i64 k = k0 + a_k + q;
      ra[q] = (row < M && k < K) ? A[row * K + k] : 0ull;
    }
    const i64 kb = k0 + b_k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const i64 col = n0 + b_n + q;
      rb[q] = (kb < K && col < N) ? B[kb * N + col] : 0ull;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) As[buf][a_k + q][a_r] = ra[q];
    reinterpret_cast<ulonglong2*>(&Bs[buf][b_k][b_n])[0] = make_ulonglong2(rb[0], rb[1]);
    reinterpret_cast<ulonglong2*>(&Bs[buf][b_k][b_n])[1] = make_ulonglong2(rb[2], rb[3]);
  };

  u64 acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0ull;

  fetch(0);
  stash(0);
  __syncthreads();

  for (i64 kt = 0; kt < total_tiles; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < total_tiles) fetch(kt + 1);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      u64 a[8], b[8];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const ulonglong2 av = *reinterpret_cast<const ulonglong2*>(&As[cur][kk][32 * c + 2 * ty]);
        const ulonglong2 bv = *reinterpret_cast<const ulonglong2*>(&Bs[cur][kk][32 * c + 2 * tx]);
        a[2 * c] = av.x;
        a[2 * c + 1] = av.y;
        b[2 * c] = bv.x;
        b[2 * c + 1] = bv.y;
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
    }
    if (kt + 1 < total_tiles) stash(cur ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const i64 row = m0 + frag_idx(i, ty);
    if (row >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const i64 col = n0 + frag_idx(j, tx);
      if (col >= N) continue;
      const i64 idx = gemm_out_index(row, col, M, N, g.hw_out);
      u64 v = acc[i][j];
      if (job.C) v += job.C[idx];
      if (g.trunc_bits > 0) v = sar(v, g.trunc_bits);
      job.Z[idx] = v;
    }
  }
}

}  // namespace

int launch_gemm_plain(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.njobs <= 0) return MPC_OK;
  const i64 gy = ceil_div(g.M, BM), gx = ceil_div(g.N, BN);
  if (gy > 65535) return fail(MPC_EINVAL, "M = %lld too large for the plain engine", (long long)g.M);
  if (gx > 0x7fffffff) return fail(MPC_EINVAL, "N too large");
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)g.njobs);
  KernelTimer timer("gemm_plain", s);
  gemm_plain_kernel<<<grid, kThreads, 0, s>>>(g);
  return check_launch("gemm_plain");
}

}  // namespace mpc
