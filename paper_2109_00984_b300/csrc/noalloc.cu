// Beaver matmul without a caller workspace: the scratch lives in a fixed-size
// device array owned by this library.
//
// Who needs this: callers that cannot allocate device memory when they call
// the library and cannot carry a workspace for it either, for example a host
// program whose device memory is entirely pre-reserved by another framework's
// pool, or code that runs where allocation calls are not allowed.  This entry
// point allocates nothing: it calls no cudaMalloc, cudaFree or allocating
// library routine.
//
// The scratch is a file-scope static __device__ array of
// MPC_NOALLOC_SCRATCH_WORDS 64-bit words (8 MiB).  Every device that loads
// the library holds it until the process exits.  In host code the array's
// name is only a host-side stand-in, so its device address is looked up once
// per device, with that device current, by the first call on that device
// (cudaGetSymbolAddress); make that first call before any stream capture.
// All calls share the one array and it keeps the last call's contents; every
// word a call reads is written by that same call first, so nothing needs
// clearing.  Calls whose kernels overlap on the GPU (two streams, or two host
// threads) race on the array: serialise them.
#include <mutex>

#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

namespace {

static __device__ __align__(256) u64 g_noalloc_scratch[MPC_NOALLOC_SCRATCH_WORDS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
u64* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
int noalloc_scratch(u64** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(MPC_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(MPC_EUNSUPPORTED, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(MPC_ECUDA, "scratch address lookup: %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = static_cast<u64*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MPC_OK;
}

// out[i] = sum_p (X_p[i] - A_p[i]); if G: G[i] = B0[i] + out[i].
__global__ void __launch_bounds__(256) noalloc_open_kernel(int P, i64 n, const u64* __restrict__ X,
                                                           const u64* __restrict__ A,
                                                           u64* __restrict__ out,
                                                           const u64* __restrict__ B0,
                                                           u64* __restrict__ G) {
  for (i64 i = blockIdx.x * (i64)blockDim.x + threadIdx.x; i < n;
       i += (i64)gridDim.x * blockDim.x) {
    u64 e = 0;
    for (int p = 0; p < P; ++p) e += X[(i64)p * n + i] - A[(i64)p * n + i];
    out[i] = e;
    if (G) G[i] = B0[i] + e;
  }
}

inline i64 round_words(i64 n) { return (n + 31) & ~(i64)31; }  // 256-byte regions

}  // namespace

}  // namespace mpc

using namespace mpc;

extern "C" int mpc_beaver_matmul_noalloc(int P, int64_t M, int64_t N, int64_t K,
                                         const uint64_t* X, const uint64_t* Y, const uint64_t* A,
                                         const uint64_t* B, const uint64_t* C, uint64_t* Z,
                                         int trunc_bits, void* stream) {
  MPC_CHECK_PARTIES(P);
  MPC_REQUIRE(M >= 0 && N >= 0 && K >= 0, "negative dimension");
  MPC_REQUIRE(trunc_bits >= 0 && trunc_bits <= 63, "trunc_bits %d outside [0, 63]", trunc_bits);
  if (M == 0 || N == 0) return MPC_OK;
  // With K = 0 the operands and a, b are empty (never read) and may be NULL.
  MPC_REQUIRE(C && Z && (K == 0 || (X && Y && A && B)), "null pointer");
  // Scratch: E [M][K], F [K][N], G = B_0 + F [K][N].  The dimensions are
  // bounded against the scratch size first, so that M*K and K*N below cannot
  // wrap: with K > 0, M*K <= W needs M <= W / K and 2*K*N <= W needs
  // N <= W / (2K).  K = 0 needs no scratch (Z = C, truncated).
  constexpr i64 W = MPC_NOALLOC_SCRATCH_WORDS;
  if (K > W || (K > 0 && (M > W / K || N > W / (2 * K))))
    return fail(MPC_ENOMEM,
                "mpc_beaver_matmul_noalloc: M=%lld N=%lld K=%lld needs more than the fixed "
                "scratch of %lld words",
                (long long)M, (long long)N, (long long)K, (long long)W);
  const i64 need = round_words(M * K) + 2 * round_words(K * N);
  if (need > W)
    return fail(MPC_ENOMEM,
                "mpc_beaver_matmul_noalloc: needs M*K + 2*K*N = %lld scratch words (each "
                "region rounded up to 32), the fixed scratch holds %lld",
                (long long)need, (long long)W);
  // M*N stays unbounded by the scratch; it indexes the caller's C and Z.
  if (!mul_fits(M, N))
    return fail(MPC_EUNSUPPORTED, "mpc_beaver_matmul_noalloc: M*N exceeds 2^52 words");
  u64* scratch = nullptr;
  if (int rc = noalloc_scratch(&scratch)) return rc;
  u64* E = scratch;
  u64* F = E + round_words(M * K);
  u64* G = F + round_words(K * N);
  cudaStream_t s = as_stream(stream);
  if (K > 0) {
    noalloc_open_kernel<<<grid_for(M * K, 256), 256, 0, s>>>(P, M * K, (const u64*)X,
                                                             (const u64*)A, E, nullptr, nullptr);
    if (int rc = check_launch("noalloc open E")) return rc;
    noalloc_open_kernel<<<grid_for(K * N, 256), 256, 0, s>>>(P, K * N, (const u64*)Y,
                                                             (const u64*)B, F, (const u64*)B, G);
    if (int rc = check_launch("noalloc open F")) return rc;
  }
  GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.hw_out = 0;
  g.trunc_bits = trunc_bits;
  g.njobs = P;
  for (int p = 0; p < P; ++p) {
    g.jobs[p].A1 = E;
    g.jobs[p].B1 = p == 0 ? G : (const u64*)B + (i64)p * K * N;
    g.jobs[p].A2 = (const u64*)A + (i64)p * M * K;
    g.jobs[p].B2 = F;
    g.jobs[p].C = (const u64*)C + (i64)p * M * N;
    g.jobs[p].Z = (u64*)Z + (i64)p * M * N;
  }
  const int rc = launch_gemm_plain(g, s);
  // The same protocol accounting as mpc_beaver_matmul: one round, E and F
  // opened, the triple's words consumed, P GEMMs of two operand pairs.
  if (rc == MPC_OK)
    stats_add(1, 8ull * (uint64_t)(M * K + K * N), 0, (uint64_t)P * (M * K + K * N + M * N),
              (uint64_t)P * 2ull * M * N * K);
  return rc;
}
