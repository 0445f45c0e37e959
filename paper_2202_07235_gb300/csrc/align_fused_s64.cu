// Instantiations of the fused scoring kernel for Q = 128 (Q/2 = 64 slots).
#include "align_fused.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_fused_s64(int HP, const FusedParams& p, cudaStream_t stream) {
  return launch_fused_s<64>(HP, p, stream);
}
}  // namespace rsvd
