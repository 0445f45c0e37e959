// rsvd_align_best: dispatch between the fused kernel (Q in {128, 256, 512})
// and the generic per-pair kernel.
#include <math.h>

#include <stdlib.h>
#include <string.h>

#include "align_ws.cuh"
#include "operand.cuh"

namespace rsvd {
namespace {

int padded_h(int H) {
  const int opts[] = {8, 12, 16, 24, 32, 64};
  for (int v : opts)
    if (H <= v) return v;
  return -1;
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_align_best(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                               float inv_sigma2, float* best, int32_t* arg, float* lse, void* stream) {
  using namespace rsvd;
  if (precision != RSVD_FP32) {
    int rc = check_tc_args(cA, N_A, T, cB, N_B, H, Q, precision);
    if (rc != RSVD_OK) return rc;
    if (!best || !arg) return RSVD_EINVAL;
    if (lse && !(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
    return align_tc(cA, N_A, T, cB, N_B, H, Q, precision, inv_sigma2, best, arg, lse, nullptr,
                    static_cast<cudaStream_t>(stream));
  }
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if (!best || !arg) return RSVD_EINVAL;
  if (lse && !(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  FusedParams p{};
  p.cA = static_cast<const float2*>(cA);
  p.cB = static_cast<const float2*>(cB);
  p.best = best;
  p.arg = arg;
  p.lse = lse;
  p.status = status_word();
  p.N_A = N_A;
  p.T = T;
  p.N_B = N_B;
  p.H = H;
  p.inv_sigma2 = inv_sigma2;
  const int HP = padded_h(H);
  // RSVD_ALIGN_KERNEL=fused selects the single-role fused kernel where the
  // warp-specialised one would be used (for cross-checks and measurements)
  const char* pick = getenv("RSVD_ALIGN_KERNEL");
  const bool classic = pick && strcmp(pick, "fused") == 0;
  rc = RSVD_EUNSUPPORTED;
  if (HP > 0) {
    if (Q == 256 && !classic) rc = launch_ws_s128(HP, p, st);
    if (Q == 512 && !classic) rc = launch_ws_s256(HP, p, st);
    if (rc == RSVD_EUNSUPPORTED) {
      if (Q == 128) rc = launch_fused_s64(HP, p, st);
      else if (Q == 256) rc = launch_fused_s128(HP, p, st);
      else if (Q == 512) rc = launch_fused_s256(HP, p, st);
    }
  }
  if (rc == RSVD_EUNSUPPORTED) rc = align_best_pairwise(cA, N_A, T, cB, N_B, H, Q, inv_sigma2, best, arg, lse, st);
  return rc;
}

// Forces the generic per-pair path (used to cross-check the fused kernel).
extern "C" int rsvd_align_best_pairwise(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                        int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                                        void* stream) {
  using namespace rsvd;
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if (!best || !arg) return RSVD_EINVAL;
  if (lse && !(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
  return align_best_pairwise(cA, N_A, T, cB, N_B, H, Q, inv_sigma2, best, arg, lse, static_cast<cudaStream_t>(stream));
}
