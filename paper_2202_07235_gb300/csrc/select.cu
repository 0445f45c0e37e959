// rsvd_select_pairs: per image, the `keep` templates with the largest coarse
// score, as (image, template) pairs for a refinement pass (the
// principal-mode-marching of the discussion, section 5: a coarse landscape at a
// low rank H, then the promising candidates recomputed at a higher rank).
//
// One warp per image. Pass i finds the largest entry that ranks below the one
// chosen in pass i - 1 in the order (score descending, template index
// ascending), so equal scores are taken in index order and no entry is chosen
// twice.
#include <math.h>

#include "rsvd_internal.cuh"

namespace rsvd {
namespace {

constexpr int kSelThreads = 256;

// (v, j) ranks before (w, k): larger score, or equal score and smaller index.
__device__ __forceinline__ bool ranks_before(float v, int j, float w, int k) { return v > w || (v == w && j < k); }

__global__ void __launch_bounds__(kSelThreads) select_kernel(const float* __restrict__ best, int N_A, int N_B, int keep,
                                                             int32_t* __restrict__ pairs) {
  const int warp = (blockIdx.x * kSelThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N_A) return;
  const float* row = best + (size_t)warp * N_B;
  float pv = INFINITY;  // previous choice (score, index); everything ranks below (+inf, -1)
  int pj = -1;
  for (int i = 0; i < keep; ++i) {
    float bv = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < N_B; j += 32) {
      const float v = row[j];
      if (ranks_before(pv, pj, v, j) && ranks_before(v, j, bv, bj)) {
        bv = v;
        bj = j;
      }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
      if (ranks_before(ov, oj, bv, bj)) {
        bv = ov;
        bj = oj;
      }
    }
    if (lane == 0) {
      pairs[2 * ((size_t)warp * keep + i)] = warp;
      pairs[2 * ((size_t)warp * keep + i) + 1] = bj;
    }
    pv = bv;
    pj = bj;
  }
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_select_pairs(const float* best, int N_A, int N_B, int keep, int32_t* pairs, void* stream) {
  using namespace rsvd;
  if (!best || !pairs || N_A <= 0 || N_B <= 0 || keep <= 0) return RSVD_EINVAL;
  if (keep > N_B || keep > 64) return RSVD_EUNSUPPORTED;
  const long long warps = N_A;
  const long long blocks = (warps * 32 + kSelThreads - 1) / kSelThreads;
  if (blocks > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
  select_kernel<<<(unsigned)blocks, kSelThreads, 0, static_cast<cudaStream_t>(stream)>>>(best, N_A, N_B, keep, pairs);
  return launch_status();
}
