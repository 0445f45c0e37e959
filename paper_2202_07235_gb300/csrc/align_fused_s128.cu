// Instantiations of the fused scoring kernel for Q = 256 (Q/2 = 128 slots).
#include "align_fused.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_fused_s128(int HP, const FusedParams& p, cudaStream_t stream) {
  return launch_fused_s<128>(HP, p, stream);
}
}  // namespace rsvd
