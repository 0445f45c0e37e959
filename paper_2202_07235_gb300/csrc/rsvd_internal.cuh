// Internal helpers shared by the CUDA translation units of librsvd.
// Not part of the ABI (symbols here have hidden visibility).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rsvd.h"

#define RSVD_HIDDEN __attribute__((visibility("hidden")))

namespace rsvd {

constexpr int kMaxR = 256;
constexpr int kMaxH = 64;
constexpr int kMaxT = 64;
constexpr int kMinQ = 16;
constexpr int kMaxQ = 1024;

// Device status word of the current device (first failure wins). Defined in abi.cu.
RSVD_HIDDEN int* status_word();

// Device-side codes recorded in the status word.
enum DeviceCode : int { kDevOk = 0, kDevBounds = 1, kDevTimeout = 2, kDevNoConverge = 3 };

__device__ __forceinline__ void record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

inline bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

inline int check_grid(int R, int Q, int H) {
  if (R <= 0 || Q <= 0 || H <= 0) return RSVD_EINVAL;
  if (!is_pow2(Q) || Q < kMinQ || Q > kMaxQ) return RSVD_EUNSUPPORTED;
  if (R > kMaxR || H > kMaxH) return RSVD_EUNSUPPORTED;
  if (H > R) return RSVD_EINVAL;
  return RSVD_OK;
}

inline int launch_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RSVD_OK : RSVD_ECUDA;
}

// ---------------------------------------------------------------------------
// Small complex helpers (float2 = re, im).
// ---------------------------------------------------------------------------
// Complex add / subtract as one packed FP32x2 instruction (sm_100+), same
// IEEE round-to-nearest result per component as two scalar adds.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i
__device__ __forceinline__ float2 cmul_mi(float2 a) { return make_float2(a.y, -a.x); }

// cos / sin of 2 pi k / 32 for k = 0..31, as exact decimal constants of the
// unit circle (cos(pi/16) etc.). Used to build compile-time twiddles
// W_N^k = exp(-2 pi i k / N) for N dividing 32.
__host__ __device__ constexpr float unit_cos32(int k) {
  constexpr float c[9] = {1.0f,
                          0.98078528040323044913f,
                          0.92387953251128675613f,
                          0.83146961230254523708f,
                          0.70710678118654752440f,
                          0.55557023301960222474f,
                          0.38268343236508977173f,
                          0.19509032201612826785f,
                          0.0f};
  // reduce k in [0, 32) to the first quadrant
  return (k <= 8) ? c[k] : (k <= 16) ? -c[16 - k] : (k <= 24) ? -c[k - 16] : c[32 - k];
}
__host__ __device__ constexpr float unit_sin32(int k) { return unit_cos32((k + 24) & 31); }

// W_N^k = exp(-2 pi i k / N), N | 32, k taken mod N.
template <int N>
__device__ __forceinline__ constexpr float2 twiddle(int k) {
  static_assert(32 % N == 0, "N must divide 32");
  return make_float2(unit_cos32(((k % N + N) % N) * (32 / N)), -unit_sin32(((k % N + N) % N) * (32 / N)));
}

// In-register DFT of length N (power of two, N <= 32):
// x[k] <- sum_n x[n] exp(-+2 pi i n k / N) (minus sign unless kInv). Radix-2
// decimation in time on a bit-reversed copy; every index and twiddle is a
// compile-time constant.
template <int N, bool kInv = false>
struct RegDft {
  static constexpr int kLog2 = (N <= 1) ? 0 : 1 + RegDft<N / 2>::kLog2;
  static __device__ __forceinline__ int brev(int i) {
    int r = 0;
#pragma unroll
    for (int b = 0; b < kLog2; ++b) r |= ((i >> b) & 1) << (kLog2 - 1 - b);
    return r;
  }
  static __device__ __forceinline__ void run(float2 (&x)[N]) {
    float2 y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = x[brev(i)];
#pragma unroll
    for (int half = 1; half < N; half *= 2) {
#pragma unroll
      for (int base = 0; base < N; base += 2 * half) {
#pragma unroll
        for (int j = 0; j < half; ++j) {
          float2 w = twiddle<N>(j * (N / (2 * half)));
          if (kInv) w.y = -w.y;
          float2 a = y[base + j];
          float2 b = y[base + j + half];
          float2 bw;
          if (j == 0) {
            bw = b;
          } else if (2 * j == half) {  // W = -i (forward) or +i (inverse)
            bw = kInv ? make_float2(-b.y, b.x) : cmul_mi(b);
          } else {
            bw = cmul(b, w);
          }
          y[base + j] = cadd(a, bw);
          y[base + j + half] = csub(a, bw);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = y[i];
  }
};
template <bool kInv>
struct RegDft<1, kInv> {
  static constexpr int kLog2 = 0;
  static __device__ __forceinline__ void run(float2 (&)[1]) {}
};

// Order-preserving map of a float to uint32 (larger float -> larger key).
__device__ __forceinline__ uint32_t ordered_key(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

}  // namespace rsvd
