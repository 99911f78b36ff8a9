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

// Implicit im2col for the B operand of a convolution (limb engine only): the
// (k, n) element of B1 is sum_{q < n1} (src1 - sub1)[q * stride1 + pos(k, n)]
// and that of B2 for job j is src2[j][pos(k, n)], where pos is the data
// position of kernel tap k = (ci, r, s) for output column n = (b, oh, ow),
// and the element is 0 in the padding.  sub1 may be null.
struct ConvGather {
  mpc_conv_desc d;
  i64 ho, wo;
  const u64* src1;
  const u64* sub1;
  i64 stride1;
  int n1;
  const u64* src2[MPC_MAX_PARTIES];
};

// splits > 1 partitions the (pair-concatenated) K range over `splits` CTAs per
// output tile; each writes its raw partial sum to partial[split][job][M][N]
// and gemm_reduce() forms Z = trunc(C + sum of partials) (exact mod 2^64).
struct GemmArgs {
  i64 M, N, K;
  i64 hw_out;
  int trunc_bits;
  int njobs;
  int splits;
  // With split-K, leave the raw partial sums in `partial` for the caller to
  // reduce (launch_relu_from_partials) instead of running gemm_reduce.
  int defer_reduce;
  u64* partial;
  const ConvGather* gather;  // host pointer; when set, B1/B2 are implicit im2col (limb only)
  // With gather and one operand pair: `gather` points to njobs convolutions,
  // job j's B1 gathered from gather[j].src2[0] (no opening) and its K =
  // c_in kh kw of gather[j].d (at most K; M and N are every job's), instead of
  // every job sharing the opened gather (the dealer's products of a batch of
  // triples).
  int gather_per_job;
  // At most this many splits (0: no cap), e.g. the shortest per-job K's sub-steps.
  int max_splits;
  // Limb engine, convolution with gather only: digit planes cut ahead of the
  // call by limb_conv_prepare (layout in its comment).  The A operands and
  // every job's B2 are taken from there; only the opened gather B1 is cut in
  // the call.  jobs[j].A1 / A2 / B2 are then unused.
  const void* prep;
  // With prep: 2 (default 0 means 2) for the layout above; 1 for prepared
  // products: prep holds only job j's A1 planes (plane set j), the products
  // A_p F having been added into C by the preparation, so each job is one pair
  // (its A1 planes times the opened gather B1).
  int prep_pairs;
  GemmJob jobs[MPC_MAX_PARTIES];
};

// Number of SMs the split heuristics plan for (B300).
constexpr int kPlanSMs = 148;

// Split count minimising waves x K-units per CTA for `tiles` output tiles and
// `units` K-units (each at least `min_units` per split).
int choose_splits(i64 tiles, i64 units, i64 min_units);

// Per-engine split choice (deterministic in the shape) and partial-sum bytes.
int plain_splits(i64 M, i64 N, i64 K, int npairs, int njobs);
// batch: a batch of one-pair products dealt beside the online phase (per-job
// gathers), split into fewer, longer pieces.
int limb_splits(i64 M, i64 N, i64 K, int npairs, int njobs, bool batch = false);
inline size_t partial_bytes(int splits, int njobs, i64 M, i64 N) {
  return splits > 1 ? (size_t)splits * njobs * M * N * sizeof(u64) : 0;
}

// Z[job] = trunc(C[job] + sum_s partial[s][job]) with the output scatter.
int gemm_reduce(const GemmArgs& g, cudaStream_t s);

__host__ __device__ __forceinline__ i64 gemm_out_index(i64 row, i64 col, i64 M, i64 N,
                                                       i64 hw_out) {
  return hw_out ? ((col / hw_out) * M + row) * hw_out + (col % hw_out) : row * N + col;
}

// Engines: each returns MPC_OK or an mpc_status with the error message set.
int launch_gemm_plain(const GemmArgs& g, cudaStream_t s);

// One product of a batched Beaver matmul, as stored in device memory.  Per
// party p the plain engine computes Z_p = C_p + E (B_p or G for p = 0) + A_p F.
struct BatchProd {
  i64 M, N, K;
  i64 tile_base;  // first work item of this product (prefix over the batch)
  i64 tiles;      // P * tiles_m * tiles_n
  i64 open_base;  // first element of this product in the batched opening
  int tiles_m, tiles_n;
  const u64 *X, *Y, *A, *B, *C;
  u64* Z;
  u64 *E, *F, *G;  // opened E [M][K], F [K][N], G = B_0 + F (workspace)
};

// Persistent plain engine over the products of `tbl` (device); `counter`
// (device, zeroed by the caller) hands out work items.
int launch_gemm_plain_batched(const BatchProd* tbl, int count, int P, int trunc_bits,
                              unsigned long long* counter, int ctas, cudaStream_t s);
int plain_tiles(i64 M, i64 N, i64* tm, i64* tn);

// Limb engine (tcgen05).  ws/ws_bytes: caller workspace (digit planes);
// limb_workspace_bytes tells how much it needs for the given shape and job
// count.  Partial sums for split-K live in g.partial (sized by the caller).
size_t limb_workspace_bytes(i64 M, i64 N, i64 K, int npairs, int njobs);
int launch_gemm_limb(const GemmArgs& g, void* ws, size_t ws_bytes, cudaStream_t s);

// The input-independent digit planes of a P-party Beaver convolution on the
// limb engine (M = c_out, K = c_in kh kw, N = batch ho wo): the planes of the
// P + 1 weight-side sources asrc = G = B_0 + F, B_1 .. B_{P-1}, F ([M][K]
// row-major operands of the GEMM's A side), then those of im2col(A_p) for
// p = 0 .. P-1 (B side, gathered from cg.src2), each plane set
// al256(16 rows K1p) bytes, K1p = K rounded up to 16.  prep must hold
// limb_conv_prep_bytes(P, M, N, K) bytes.
size_t limb_conv_prep_bytes(int P, i64 M, i64 N, i64 K);
int limb_conv_prepare(int P, const ConvGather& cg, i64 M, i64 N, i64 K,
                      const u64* const* asrc, void* prep, cudaStream_t s);
bool limb_supported(i64 M, i64 N, i64 K);

// The digit planes of n row-major [M][K] sources src[i] into out, one plane set
// of al256(16 M K1p) bytes per source (K1p = K rounded up to 16), in order.
int limb_cut_planes_a(int n, const u64* const* src, i64 M, i64 K, void* out, cudaStream_t s);
size_t limb_planes_a_bytes(i64 M, i64 K);

// Grouped limb engine: the Beaver products of a batch in one digit-plane launch
// (which also opens E and F) and one persistent GEMM launch.  Per product and
// party p:
//   Z_p = trunc(C_p + E G_p + A_p F),  E = sum_q (X_q - A_q), F = sum_q (Y_q - B_q),
//   G_0 = B_0 + F, G_p = B_p (p >= 1),
// with X, A [P][M][K], Y, B [P][K][N], C and Z [P][M][N] (device).  Products
// are processed in the order given: put the longest K first so that the
// persistent CTAs finish together.
struct GroupedProduct {
  i64 M, N, K;
  const u64 *X, *Y, *A, *B, *C;
  u64* Z;
};
size_t limb_grouped_workspace_bytes(int P, int count, const GroupedProduct* prods);
// ctas: persistent CTAs (0 = one per SM).
int launch_gemm_limb_grouped(int P, int count, const GroupedProduct* prods, int trunc_bits,
                             int ctas, void* ws, size_t ws_bytes, cudaStream_t s);

// Engine dispatch shared by the entry points: split choice, workspace bytes
// (split-K partials, then limb planes) and the launch of one GEMM job set.
int engine_splits(int algo, i64 M, i64 N, i64 K, int npairs, int njobs, bool batch = false);
size_t engine_ws(int algo, i64 M, i64 N, i64 K, int npairs, int njobs, bool batch = false);
// used (optional): the job set as launched (split count, partial buffer).
int run_gemm(GemmArgs g, int algo, void* ws, size_t ws_bytes, cudaStream_t s,
             GemmArgs* used = nullptr);

// Two-party fused private ReLU (dealer regenerated in registers, material at op
// .. op + 3, as mpc_private_relu_fused) of a GEMM job set's output without
// materialising it: element i of party p is trunc(C_p[i] + sum over splits of
// the partial sums at the GEMM position of output index i), or Z_p[i] when
// the job set was not split.  Y [2][M N] receives the ReLU.  Requires njobs = 2.
// S (may be null): two-party shares [2][M N] added to each truncated output
// before the ReLU (a residual connection).
int launch_relu_of_gemm(const GemmArgs& g, u64* Y, u64 seed, u64 op, cudaStream_t s,
                        const u64* S = nullptr);

}  // namespace mpc
