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

// One thread per VEC adjacent columns of one (job, row), flattened over all
// rows so every thread has work: the partial sums are read VEC words at a
// time (16-byte loads for VEC = 2), four splits per batch of independent
// loads; one 32-bit division per element for the conv output scatter.
template <int VEC>
__global__ void __launch_bounds__(256) gemm_reduce_kernel(const GemmArgs g) {
  const i64 MN = g.M * g.N;
  const i64 nv = (g.N + VEC - 1) / VEC;
  const i64 total = g.M * g.njobs * nv;
  const i64 sstride = (i64)g.njobs * MN;
  const uint32_t hw = (uint32_t)g.hw_out;
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < total;
       i += (i64)gridDim.x * blockDim.x) {
    const i64 rj = i / nv;
    const i64 col0 = (i - rj * nv) * VEC;
    const int job = (int)(rj / g.M);
    const i64 row = rj - (i64)job * g.M;
    const u64* part = g.partial + (i64)job * MN + row * g.N + col0;
    u64 v[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) v[e] = 0;
    int s = 0;
    for (; s + 4 <= g.splits; s += 4) {
      u64 w[4][VEC];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const u64* src = part + (i64)(s + q) * sstride;
        if (VEC == 2) {
          const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(src);
          w[q][0] = t.x;
          w[q][VEC - 1] = t.y;
        } else {
          w[q][0] = src[0];
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int e = 0; e < VEC; ++e) v[e] += w[q][e];
    }
    for (; s < g.splits; ++s) {
      const u64* src = part + (i64)s * sstride;
      if (VEC == 2) {
        const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(src);
        v[0] += t.x;
        v[VEC - 1] += t.y;
      } else {
        v[0] += src[0];
      }
    }
    const u64* C = g.jobs[job].C;
    u64* Z = g.jobs[job].Z;
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const i64 col = col0 + e;
      i64 idx;
      if (hw) {
        const uint32_t b = (uint32_t)col / hw;
        idx = ((i64)b * g.M + row) * hw + ((uint32_t)col - b * hw);
      } else {
        idx = row * g.N + col;
      }
      u64 r = v[e];
      if (C) r += C[idx];
      if (g.trunc_bits > 0) r = sar(r, g.trunc_bits);
      Z[idx] = r;
    }
  }
}

}  // namespace

int gemm_reduce(const GemmArgs& g, cudaStream_t s) {
  const i64 total = g.M * g.N * g.njobs;
  if (total == 0) return MPC_OK;
  // Pairs of columns when every row starts 16-byte aligned (N even; the
  // partial buffer is 256-byte aligned).
  const bool vec2 = (g.N % 2 == 0) && ((reinterpret_cast<uintptr_t>(g.partial) & 15) == 0);
  const i64 items = vec2 ? total / 2 : total;
  const unsigned blocks = (unsigned)std::min<i64>(ceil_div(items, 256), 148 * 16);
  if (vec2)
    gemm_reduce_kernel<2><<<blocks, 256, 0, s>>>(g);
  else
    gemm_reduce_kernel<1><<<blocks, 256, 0, s>>>(g);
  return check_launch("gemm_reduce");
}

}  // namespace mpc
