// Split-K planning and the reduction of partial sums shared by both engines.
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

__global__ void __launch_bounds__(256) gemm_reduce_kernel(const GemmArgs g) {
  const i64 MN = g.M * g.N;
  const i64 total = MN * g.njobs;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const int job = (int)(i / MN);
    const i64 e = i % MN, row = e / g.N, col = e % g.N;
    u64 v = 0;
    for (int s = 0; s < g.splits; ++s) v += g.partial[((i64)s * g.njobs + job) * MN + e];
    const i64 idx = gemm_out_index(row, col, g.M, g.N, g.hw_out);
    if (g.jobs[job].C) v += g.jobs[job].C[idx];
    if (g.trunc_bits > 0) v = sar(v, g.trunc_bits);
    g.jobs[job].Z[idx] = v;
  }
}

}  // namespace

int gemm_reduce(const GemmArgs& g, cudaStream_t s) {
  const i64 total = g.M * g.N * g.njobs;
  if (total == 0) return MPC_OK;
  gemm_reduce_kernel<<<grid_for(total, 256), 256, 0, s>>>(g);
  return check_launch("gemm_reduce");
}

}  // namespace mpc
