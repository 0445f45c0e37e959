// Instantiations of the log-sum-exp gradient kernel for Q = 512.
#include "align_grad.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_grad_s256(int HP, bool tmpl, const GradParams& p, cudaStream_t stream) {
  return launch_grad_s<256>(HP, tmpl, p, stream);
}
}  // namespace rsvd
