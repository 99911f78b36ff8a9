// Ring GEMM job description shared by the plain and limb engines.
#pragma once

#include "common.cuh"

namespace mpc {

// Z = C + A1 B1 (+ A2 B2) over Z/2^64, then optionally Z = s(Z) >> trunc_bits.
// A1, A2: [M][K] row-major; B1, B2: [K][N] row-major.  A2/B2 may be null (one
// pair).  C may be null (zero).  One job per party; all jobs share M, N, K.
// Output index of (row, col): row * N + col when hw_out == 0, else the NCHW
// scatter ((col / hw_out) * M + row) * hw_out + col % hw_out (conv output with
// batch folded into the columns).  C uses the same index.
struct GemmJob {
  const u64* A1;
  const u64* B1;
  const u64* A2;
  const u64* B2;
  const u64* C;
  u64* Z;
};

struct GemmArgs {
  i64 M, N, K;
  i64 hw_out;
  int trunc_bits;
  int njobs;
  GemmJob jobs[MPC_MAX_PARTIES];
};

__host__ __device__ __forceinline__ i64 gemm_out_index(i64 row, i64 col, i64 M, i64 N,
                                                       i64 hw_out) {
  return hw_out ? ((col / hw_out) * M + row) * hw_out + (col % hw_out) : row * N + col;
}

// Engines: each returns MPC_OK or an mpc_status with the error message set.
int launch_gemm_plain(const GemmArgs& g, cudaStream_t s);

// Limb engine (tcgen05).  ws/ws_bytes: caller workspace; limb_workspace_bytes
// tells how much it needs for the given shape and job count.
size_t limb_workspace_bytes(i64 M, i64 N, i64 K, int npairs, int njobs);
int launch_gemm_limb(const GemmArgs& g, void* ws, size_t ws_bytes, cudaStream_t s);
bool limb_supported(i64 M, i64 N, i64 K);

}  // namespace mpc
