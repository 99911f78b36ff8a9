// Limb-split ring GEMM on tcgen05 tensor cores (placeholder until the engine lands).
#include "gemm.hpp"
#include "host.hpp"

namespace mpc {

bool limb_supported(i64, i64, i64) { return false; }

size_t limb_workspace_bytes(i64, i64, i64, int, int) { return 0; }

int launch_gemm_limb(const GemmArgs&, void*, size_t, cudaStream_t) {
  return fail(MPC_EUNSUPPORTED, "limb engine not built");
}

}  // namespace mpc
