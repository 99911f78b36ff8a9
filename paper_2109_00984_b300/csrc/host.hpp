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
