// Instantiations of the log-sum-exp gradient kernel for Q = 256.
#include "align_grad.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_grad_s128(int HP, bool tmpl, const GradParams& p, cudaStream_t stream) {
  return launch_grad_s<128>(HP, tmpl, p, stream);
}
}  // namespace rsvd
