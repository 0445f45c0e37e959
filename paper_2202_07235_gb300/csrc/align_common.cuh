// Helpers shared by the scoring kernels: argument checks and the running
// max / argmax / log-sum-exp reductions.
#pragma once

#include <math.h>

#include "rsvd_internal.cuh"

namespace rsvd {

inline int check_align_args(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision) {
  if (!cA || !cB) return RSVD_EINVAL;
  if (N_A <= 0 || N_B <= 0 || T <= 0 || H <= 0 || Q <= 0) return RSVD_EINVAL;
  if (!is_pow2(Q) || Q < kMinQ || Q > kMaxQ || H > kMaxH || T > kMaxT) return RSVD_EUNSUPPORTED;
  if (precision != RSVD_FP32) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)cA & 15u) || ((uintptr_t)cB & 15u)) return RSVD_EINVAL;
  if ((long long)N_A * T > 0x7fffffffLL / 2) return RSVD_EUNSUPPORTED;
  return RSVD_OK;
}

// Arguments of the tensor-core path (operand forms, operand.cuh): Q in
// {128, 256, 512}, H <= 32, T <= 64, operand planes 16-byte aligned (the row
// factors of RSVD_FP16X3 follow the planes, 16-byte aligned too).
inline int check_tc_args(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision) {
  if (!cA || !cB) return RSVD_EINVAL;
  if (N_A <= 0 || N_B <= 0 || T <= 0 || H <= 0 || Q <= 0) return RSVD_EINVAL;
  if (precision != RSVD_BF16 && precision != RSVD_FP16 && precision != RSVD_BF16X3 && precision != RSVD_FP16X3)
    return RSVD_EUNSUPPORTED;
  if (!(Q == 128 || Q == 256 || Q == 512) || H > 32 || T > kMaxT) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)cA & 15u) || ((uintptr_t)cB & 15u)) return RSVD_EINVAL;
  if ((long long)N_A * T > 0x7fffffffLL / 2) return RSVD_EUNSUPPORTED;
  return RSVD_OK;
}

// Running log-sum-exp state (m, s): the represented value is m + log(s).
__device__ __forceinline__ void lse_push(float& m, float& s, float v) {
  if (v > m) {
    s = s * __expf(m - v) + 1.0f;
    m = v;
  } else {
    s += __expf(v - m);
  }
}

__device__ __forceinline__ void lse_merge(float& m, float& s, float m2, float s2) {
  if (!(s2 > 0.0f)) return;
  if (!(s > 0.0f)) {
    m = m2;
    s = s2;
    return;
  }
  if (m2 > m) {
    s = s * __expf(m - m2) + s2;
    m = m2;
  } else {
    s += s2 * __expf(m2 - m);
  }
}

// Max with the smallest index among equal values, over `width` consecutive lanes.
__device__ __forceinline__ void argmax_warp_reduce(float& v, int& i, int width) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off < width) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, off, width);
      const int oi = __shfl_xor_sync(0xffffffffu, i, off, width);
      if (ov > v || (ov == v && oi < i)) {
        v = ov;
        i = oi;
      }
    }
  }
}

__device__ __forceinline__ void lse_warp_reduce(float& m, float& s, int width) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (off < width) {
      const float om = __shfl_xor_sync(0xffffffffu, m, off, width);
      const float os = __shfl_xor_sync(0xffffffffu, s, off, width);
      lse_merge(m, s, om, os);
    }
  }
}

// Max and first-index argmax of N values given in increasing index order, as a
// pairwise tree (depth log2 N): at each node the right child wins only if
// strictly larger, so equal values keep the smaller index.
template <int N>
__device__ __forceinline__ void tree_argmax(const float (&v)[N], float& best, int& idx) {
  static_assert((N & (N - 1)) == 0, "N must be a power of two");
  float bv[N];
  int bi[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    bv[i] = v[i];
    bi[i] = i;
  }
#pragma unroll
  for (int w = 1; w < N; w *= 2) {
#pragma unroll
    for (int i = 0; i < N; i += 2 * w) {
      const bool right = bv[i + w] > bv[i];
      bv[i] = right ? bv[i + w] : bv[i];
      bi[i] = right ? bi[i + w] : bi[i];
    }
  }
  best = bv[0];
  idx = bi[0];
}

// Pairwise-tree sum of N values.
template <int N>
__device__ __forceinline__ float tree_sum(float (&v)[N]) {
#pragma unroll
  for (int w = 1; w < N; w *= 2)
#pragma unroll
    for (int i = 0; i < N; i += 2 * w) v[i] += v[i + w];
  return v[0];
}

// Tensor-core path for the operand forms (align_tc.cu): best/arg/lse, or X when X != NULL.
RSVD_HIDDEN int align_tc(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                         float inv_sigma2, float* best, int32_t* arg, float* lse, float* X, cudaStream_t stream);

// Generic per-pair path (align_pair.cu).
RSVD_HIDDEN int align_best_pairwise(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                    float inv_sigma2, float* best, int32_t* arg, float* lse, cudaStream_t stream);

}  // namespace rsvd
