// Instantiations of the log-sum-exp gradient kernel for Q = 128.
#include "align_grad.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_grad_s64(int HP, bool tmpl, const GradParams& p, cudaStream_t stream) {
  return launch_grad_s<64>(HP, tmpl, p, stream);
}
}  // namespace rsvd
