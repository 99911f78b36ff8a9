// Split-K planning and the reduction of partial sums shared by both engines.
#include <algorithm>
#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

int choose_splits(i64 tiles, i64 units, i64 min_units) {
  if (tiles <= 0 || units <= 0) return 1;
  int best = 1;
  i64 best_cost = ceil_div(tiles, kPlanSMs) * units;
  for (int s = 2; s <= 64; ++s) {
    const i64 per = ceil_div(units, s);
    if (per < min_units) break;
    if (tiles * s > 65535) break;
    const i64 cost = ceil_div(tiles * s, kPlanSMs) * per;
    if (cost * 100 < best_cost * 97) {  // demand a 3% gain per extra split level
      best = s;
      best_cost = cost;
    }
  }
  return best;
}

namespace {

// Rows (job, row) on the y grid, columns on threads: coalesced partial reads,
// one 32-bit division per element for the conv output scatter.
__global__ void __launch_bounds__(256) gemm_reduce_kernel(const GemmArgs g) {
  const i64 MN = g.M * g.N;
  const i64 rows = g.M * g.njobs;
  const uint32_t hw = (uint32_t)g.hw_out;
  for (i64 rj = blockIdx.y; rj < rows; rj += gridDim.y) {
    const int job = (int)(rj / g.M);
    const i64 row = rj - (i64)job * g.M;
    const u64* part = g.partial + (i64)job * MN + row * g.N;
    const u64* C = g.jobs[job].C;
    u64* Z = g.jobs[job].Z;
    for (i64 col = blockIdx.x * (i64)blockDim.x + threadIdx.x; col < g.N;
         col += (i64)gridDim.x * blockDim.x) {
      u64 v = 0;
      for (int s = 0; s < g.splits; ++s) v += part[(i64)s * g.njobs * MN + col];
      i64 idx;
      if (hw) {
        const uint32_t b = (uint32_t)col / hw;
        idx = ((i64)b * g.M + row) * hw + ((uint32_t)col - b * hw);
      } else {
        idx = row * g.N + col;
      }
      if (C) v += C[idx];
      if (g.trunc_bits > 0) v = sar(v, g.trunc_bits);
      Z[idx] = v;
    }
  }
}

}  // namespace

int gemm_reduce(const GemmArgs& g, cudaStream_t s) {
  const i64 total = g.M * g.N * g.njobs;
  if (total == 0) return MPC_OK;
  const i64 rows = g.M * g.njobs;
  const unsigned gx = (unsigned)std::min<i64>(ceil_div(g.N, 256), 64);
  const unsigned gy = (unsigned)std::min<i64>(rows, 65535);
  gemm_reduce_kernel<<<dim3(gx, gy), 256, 0, s>>>(g);
  return check_launch("gemm_reduce");
}

}  // namespace mpc
