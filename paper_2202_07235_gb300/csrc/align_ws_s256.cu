// Instantiations of the warp-specialised scoring kernel for Q = 512.
#include "align_ws.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_ws_s256(int HP, const FusedParams& p, cudaStream_t stream) {
  switch (HP) {
    case 8: return launch_ws_cfg<256, 8>(p, stream);
    case 12: return launch_ws_cfg<256, 12>(p, stream);
    case 16: return launch_ws_cfg<256, 16>(p, stream);
    default: return RSVD_EUNSUPPORTED;
  }
}
}  // namespace rsvd
