// Host-side helpers shared by the entry points: error reporting, counters.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpc_ring.h"

namespace mpc {

// Records a formatted message as the calling thread's last error, returns code.
int fail(int code, const char* fmt, ...);

// MPC_OK if the last launch on this thread succeeded, else MPC_ECUDA + message.
int check_launch(const char* what);

// Adds to the process-wide protocol counters (thread-safe).
void stats_add(uint64_t rounds, uint64_t bytes_opened, uint64_t and_gates,
               uint64_t triple_words, uint64_t ring_macs);

// Device address of the current device's status word (nullptr + message on error).
int* device_status_ptr();

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Size guard, applied before any size arithmetic on a caller's shape.  Every
// workspace formula of the library is a handful of terms M*K, K*N, M*N (or a
// convolution's data size) times 8 bytes and at most 2 * MPC_MAX_PARTIES, so
// with each such product at most kMaxWords = 2^52 words no formula can wrap
// 64 bits.  mul_fits(a, b): a, b >= 0 and a * b <= kMaxWords, tested without
// forming the product.
constexpr long long kMaxWords = 1ll << 52;
inline bool mul_fits(long long a, long long b) {
  return a >= 0 && b >= 0 && (a == 0 || b <= kMaxWords / a);
}
inline bool gemm_shape_fits(long long M, long long N, long long K) {
  return mul_fits(M, K) && mul_fits(K, N) && mul_fits(M, N);
}

// Optional per-kernel timing (mpc_profile_enable): brackets one launch with a
// pair of CUDA events on its stream when profiling is on, a no-op otherwise.
class KernelTimer {
 public:
  KernelTimer(const char* name, cudaStream_t s);
  ~KernelTimer();

 private:
  int slot_;
  cudaStream_t s_;
};

}  // namespace mpc

#define MPC_REQUIRE(cond, ...)                          \
  do {                                                  \
    if (!(cond)) return ::mpc::fail(MPC_EINVAL, __VA_ARGS__); \
  } while (0)

#define MPC_CHECK_PARTIES(P) \
  MPC_REQUIRE((P) >= 1 && (P) <= MPC_MAX_PARTIES, "party count %d outside [1, %d]", (int)(P), MPC_MAX_PARTIES)

// Dispatch a template on the party count 1..8.
#define MPC_DISPATCH_P(P, FN, ...)       \
  switch (P) {                           \
    case 1: FN<1>(__VA_ARGS__); break;   \
    case 2: FN<2>(__VA_ARGS__); break;   \
    case 3: FN<3>(__VA_ARGS__); break;   \
    case 4: FN<4>(__VA_ARGS__); break;   \
    case 5: FN<5>(__VA_ARGS__); break;   \
    case 6: FN<6>(__VA_ARGS__); break;   \
    case 7: FN<7>(__VA_ARGS__); break;   \
    default: FN<8>(__VA_ARGS__); break;  \
  }
