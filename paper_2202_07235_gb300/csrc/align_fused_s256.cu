// Instantiations of the fused scoring kernel for Q = 512 (Q/2 = 256 slots).
#include "align_fused.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_fused_s256(int HP, const FusedParams& p, cudaStream_t stream) {
  return launch_fused_s<256>(HP, p, stream);
}
}  // namespace rsvd
