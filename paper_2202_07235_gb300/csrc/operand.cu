// rsvd_pack: FP32 compressed rings -> operand planes of the tensor-core path
// (layout and rounding in operand.cuh).
#include "operand.cuh"

namespace rsvd {
namespace {

// One thread per (row, h, slot) coefficient; writes are scattered over the
// plane (each 4-byte (re, im) pair lands in its tile/group/lane position).
__global__ void pack_kernel(const float2* __restrict__ c32, long long total, OperandLayout L, int precision,
                            uint16_t* out) {
  const int M = L.Q / 2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i % M);
    const long long rh = i / M;
    const int h = (int)(rh % L.H);
    const long long row = rh / L.H;
    const long long n = row / L.T;
    const int t = (int)(row % L.T);
    operand_put(out, L.plane_elems, precision, operand_index(L, n, t, h, s), c32[i]);
  }
}

// RSVD_FP16X3: one warp per operand row (object n, translation t). The warp
// finds the row's largest component magnitude m, takes e = 14 - E with
// 2^(E-1) <= m < 2^E (frexp: m = f 2^E, f in [0.5, 1)), clamped to
// [-126, 126] so that 2^-e stays a normal FP32 number (e = 0 for a zero row),
// writes the row factor 2^-e and then the half parts of x 2^e (exact scaling)
// hi = rn_fp16(x 2^e), lo = rn_fp16(x 2^e - hi) (the difference is exact in FP32).
__global__ void pack_scaled_kernel(const float2* __restrict__ c32, long long rows, OperandLayout L, uint16_t* out,
                                   float* scale) {
  const int lane = threadIdx.x & 31;
  const int M = L.Q / 2;
  const int per_row = L.H * M;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
    const float2* src = c32 + row * per_row;
    float m = 0.0f;
    for (int i = lane; i < per_row; i += 32) {
      const float2 v = src[i];
      m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int E = 0;
    (void)frexpf(m, &E);
    const int e = m > 0.0f ? max(-126, min(126, 14 - E)) : 0;
    if (lane == 0) scale[row] = ldexpf(1.0f, -e);
    const long long n = row / L.T;
    const int t = (int)(row % L.T);
    for (int i = lane; i < per_row; i += 32) {
      const float2 v = src[i];
      const int h = i / M, sl = i % M;
      const float xr = ldexpf(v.x, e), xi = ldexpf(v.y, e);
      const __half2 hi = __floats2half2_rn(xr, xi);
      const __half2 lo = __floats2half2_rn(xr - __low2float(hi), xi - __high2float(hi));
      const long long idx = operand_index(L, n, t, h, sl);
      *reinterpret_cast<__half2*>(out + idx) = hi;
      *reinterpret_cast<__half2*>(out + L.plane_elems + idx) = lo;
    }
  }
}

}  // namespace

RSVD_HIDDEN int launch_pack_operands(const float2* c32, long long N, const OperandLayout& L, int precision,
                                     uint16_t* out, cudaStream_t stream) {
  if (cudaMemsetAsync(out, 0, operand_bytes(L, precision), stream) != cudaSuccess) return RSVD_ECUDA;
  if (precision == RSVD_FP16X3) {
    const long long rows = N * L.T;
    const int threads = 256;  // 8 rows per block
    const long long want = (rows + 7) / 8;
    const int blocks = (int)(want < 152LL * 16 ? want : 152LL * 16);
    float* scale = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(out) + operand_scale_offset(L, precision));
    pack_scaled_kernel<<<blocks, threads, 0, stream>>>(c32, rows, L, out, scale);
    return launch_status();
  }
  const long long total = N * L.T * L.H * (long long)(L.Q / 2);
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 152LL * 32 ? want : 152LL * 32);
  pack_kernel<<<blocks, threads, 0, stream>>>(c32, total, L, precision, out);
  return launch_status();
}

}  // namespace rsvd

extern "C" int rsvd_pack(const void* c32, int N, int T, int H, int Q, int precision, void* out, void* stream) {
  using namespace rsvd;
  if (!c32 || !out || N <= 0 || T <= 0 || H <= 0 || Q <= 0) return RSVD_EINVAL;
  if (!is_operand_precision(precision)) return RSVD_EUNSUPPORTED;
  OperandLayout L{};
  if (!make_operand_layout(N, T, H, Q, &L)) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)c32 & 7u) || ((uintptr_t)out & 15u)) return RSVD_EINVAL;
  return launch_pack_operands(static_cast<const float2*>(c32), N, L, precision, static_cast<uint16_t*>(out),
                              static_cast<cudaStream_t>(stream));
}
