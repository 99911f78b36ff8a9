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

// One 128x128 output tile of Z = C + A1 B1 (+ A2 B2) over the pair-concatenated
// K tiles [kt_begin, kt_end).  With `part` set the raw sum is stored there
// (row-major M x N, no C, no truncation) for a later split-K reduction.
__device__ __forceinline__ void plain_tile(const GemmJob& job, i64 M, i64 N, i64 K, i64 m0,
                                           i64 n0, i64 kt_begin, i64 kt_end, i64 hw_out,
                                           int trunc_bits, u64* part,
                                           u64 (*As)[BK][BM + APAD], u64 (*Bs)[BK][BN]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // K tiles of one pair; at least 1 so that the pair split below never
  // divides by zero when K = 0 (then no tile is in range and Z = C).
  const i64 ktiles = K > 0 ? ceil_div(K, BK) : 1;

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
      ra[q] = (kt < kt_end && row < M && k < K) ? A[row * K + k] : 0ull;
    }
    const i64 kb = k0 + b_k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const i64 col = n0 + b_n + q;
      rb[q] = (kt < kt_end && kb < K && col < N) ? B[kb * N + col] : 0ull;
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

  fetch(kt_begin);
  stash(0);
  __syncthreads();

  for (i64 kt = kt_begin; kt < kt_end; ++kt) {
    const int cur = (int)((kt - kt_begin) & 1);
    if (kt + 1 < kt_end) fetch(kt + 1);
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
    if (kt + 1 < kt_end) stash(cur ^ 1);
    __syncthreads();
  }

  if (part) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const i64 row = m0 + frag_idx(i, ty);
      if (row >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const i64 col = n0 + frag_idx(j, tx);
        if (col < N) part[row * N + col] = acc[i][j];
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const i64 row = m0 + frag_idx(i, ty);
    if (row >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const i64 col = n0 + frag_idx(j, tx);
      if (col >= N) continue;
      const i64 idx = gemm_out_index(row, col, M, N, hw_out);
      u64 v = acc[i][j];
      if (job.C) v += job.C[idx];
      if (trunc_bits > 0) v = sar(v, trunc_bits);
      job.Z[idx] = v;
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) gemm_plain_kernel(const GemmArgs g) {
  __shared__ __align__(16) u64 As[2][BK][BM + APAD];
  __shared__ __align__(16) u64 Bs[2][BK][BN];
  const int job_id = blockIdx.z / g.splits, split = blockIdx.z % g.splits;
  const GemmJob& job = g.jobs[job_id];
  const int npairs = job.A2 ? 2 : 1;
  // This CTA's share of the pair-concatenated K tiles.
  const i64 all_tiles = ceil_div(g.K, BK) * npairs;
  const i64 kt_begin = all_tiles * split / g.splits;
  const i64 kt_end = all_tiles * (split + 1) / g.splits;
  u64* part = g.splits > 1 ? g.partial + ((i64)split * g.njobs + job_id) * g.M * g.N : nullptr;
  plain_tile(job, g.M, g.N, g.K, (i64)blockIdx.y * BM, (i64)blockIdx.x * BN, kt_begin, kt_end,
             g.hw_out, g.trunc_bits, part, As, Bs);
}

// Persistent batched variant: CTAs claim output tiles of many products from an
// atomic counter until the work list is exhausted.  Products are laid out in
// the table in processing order (largest K first); tile t of product i is
// party (t / (tm * tn)), row tile ((t / tn) % tm), column tile (t % tn).
__global__ void __launch_bounds__(kThreads, 1) gemm_plain_batched_kernel(
    const BatchProd* __restrict__ tbl, int count, int P, int trunc_bits,
    unsigned long long* counter) {
  __shared__ __align__(16) u64 As[2][BK][BM + APAD];
  __shared__ __align__(16) u64 Bs[2][BK][BN];
  __shared__ long long s_item;
  const long long total = tbl[count - 1].tile_base + tbl[count - 1].tiles;
  for (;;) {
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long item = s_item;
    __syncthreads();
    if (item >= total) break;
    int lo = 0, hi = count - 1;  // last product with tile_base <= item
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tbl[mid].tile_base <= item) lo = mid; else hi = mid - 1;
    }
    const BatchProd& b = tbl[lo];
    const long long local = item - b.tile_base;
    const long long per_party = (long long)b.tiles_m * b.tiles_n;
    const int p = (int)(local / per_party);
    const long long r = local % per_party;
    GemmJob job;
    job.A1 = b.E;
    job.B1 = p == 0 ? b.G : b.B + (i64)p * b.K * b.N;
    job.A2 = b.A + (i64)p * b.M * b.K;
    job.B2 = b.F;
    job.C = b.C + (i64)p * b.M * b.N;
    job.Z = b.Z + (i64)p * b.M * b.N;
    plain_tile(job, b.M, b.N, b.K, (r / b.tiles_n) * BM, (r % b.tiles_n) * BN, 0,
               2 * ceil_div(b.K, BK), 0, trunc_bits, nullptr, As, Bs);
    __syncthreads();
  }
}

}  // namespace

int launch_gemm_plain_batched(const BatchProd* tbl, int count, int P, int trunc_bits,
                              unsigned long long* counter, int ctas, cudaStream_t s) {
  if (count <= 0) return MPC_OK;
  KernelTimer timer("gemm_plain_batched", s);
  gemm_plain_batched_kernel<<<ctas, kThreads, 0, s>>>(tbl, count, P, trunc_bits, counter);
  return check_launch("gemm_plain_batched");
}

int plain_tiles(i64 M, i64 N, i64* tm, i64* tn) {
  *tm = ceil_div(M, BM);
  *tn = ceil_div(N, BN);
  return MPC_OK;
}

int plain_splits(i64 M, i64 N, i64 K, int npairs, int njobs) {
  const i64 tiles = ceil_div(M, BM) * ceil_div(N, BN) * njobs;
  return choose_splits(tiles, ceil_div(K, BK) * npairs, 32);
}

int launch_gemm_plain(const GemmArgs& g_in, cudaStream_t s) {
  GemmArgs g = g_in;
  if (g.splits < 1) g.splits = 1;  // callers that leave it zero ask for no split
  if (g.M <= 0 || g.N <= 0 || g.njobs <= 0) return MPC_OK;
  const i64 gy = ceil_div(g.M, BM), gx = ceil_div(g.N, BN);
  if (gy > 65535) return fail(MPC_EINVAL, "M = %lld too large for the plain engine", (long long)g.M);
  if (gx > 0x7fffffff) return fail(MPC_EINVAL, "N too large");
  if ((g.splits > 1 && g.partial == nullptr) || g.splits * g.njobs > 65535)
    return fail(MPC_EINVAL, "bad split configuration");
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(g.njobs * g.splits));
  {
    KernelTimer timer("gemm_plain", s);
    gemm_plain_kernel<<<grid, kThreads, 0, s>>>(g);
    if (int rc = check_launch("gemm_plain")) return rc;
  }
  return (g.splits > 1 && !g.defer_reduce) ? gemm_reduce(g, s) : MPC_OK;
}

}  // namespace mpc
