// Arithmetic-rate probes: the measured denominators of the FP32-ALU and MUFU
// rooflines. Not part of the paper's method.
//
// Each thread runs independent dependency chains of one instruction kind in
// registers (no memory traffic inside the loop), long enough that the launch
// is dominated by the loop; the caller times the launch with CUDA events on
// `stream` and divides the operation count by the elapsed time. Results are
// written to a device sink only when they equal a value the host never
// passes, so the loops cannot be removed and nothing is stored.
#include "rsvd_internal.cuh"

namespace rsvd {
namespace {

__device__ float g_rate_sink;

constexpr int kChains = 8;

// FP32 fused multiply-add, one scalar FFMA per chain step (2 flops).
__global__ void __launch_bounds__(256) ffma_rate_kernel(int iters, float seed, float never) {
  float acc[2 * kChains];
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) acc[k] = seed * (float)(threadIdx.x + k);
  const float m = 1.0f - seed * 1e-7f, c = seed * 1e-3f;
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < 2 * kChains; ++k) acc[k] = fmaf(acc[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) s += acc[k];
  if (s == never) g_rate_sink = s;
}

// Packed FP32x2 fused multiply-add (two FMAs per instruction, 4 flops).
__global__ void __launch_bounds__(256) ffma2_rate_kernel(int iters, float seed, float never) {
  float2 acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = make_float2(seed * (float)(threadIdx.x + k), seed * (float)k);
  const float2 m = make_float2(1.0f - seed * 1e-7f, 1.0f - seed * 2e-7f);
  const float2 c = make_float2(seed * 1e-3f, seed * 2e-3f);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) acc[k] = __ffma2_rn(acc[k], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k].x + acc[k].y;
  if (s == never) g_rate_sink = s;
}

// Special-function unit: base-2 exponential (ex2.approx), one per chain step.
__global__ void __launch_bounds__(256) ex2_rate_kernel(int iters, float seed, float never) {
  float acc[2 * kChains];
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) acc[k] = -seed * (float)(threadIdx.x + k + 1);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < 2 * kChains; ++k) {
        float y;
        asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(acc[k]));
        acc[k] = -y;  // stays in (-1, 0]: a bounded, data-dependent chain
      }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * kChains; ++k) s += acc[k];
  if (s == never) g_rate_sink = s;
}

}  // namespace
}  // namespace rsvd

extern "C" {

int rsvd_rate_probe(int kind, int blocks, int iters, double* ops_out, void* stream) {
  if (!ops_out || blocks <= 0 || iters <= 0 || blocks > (1 << 20)) return RSVD_EINVAL;
  const int threads = 256;
  const double steps = (double)blocks * threads * (double)iters * 4.0 * (2 * rsvd::kChains);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float seed = 0.5f, never = -12345.678f;
  switch (kind) {
    case RSVD_RATE_FFMA:
      rsvd::ffma_rate_kernel<<<blocks, threads, 0, s>>>(iters, seed, never);
      *ops_out = steps * 2.0;  // flops: 2 per FMA
      break;
    case RSVD_RATE_FFMA2:
      rsvd::ffma2_rate_kernel<<<blocks, threads, 0, s>>>(iters, seed, never);
      *ops_out = steps * 2.0;  // kChains packed chains x 2 lanes = 2 kChains FMAs per step
      break;
    case RSVD_RATE_EX2:
      rsvd::ex2_rate_kernel<<<blocks, threads, 0, s>>>(iters, seed, never);
      *ops_out = steps;  // exponentials
      break;
    default:
      return RSVD_EINVAL;
  }
  return rsvd::launch_status();
}

}  // extern "C"
