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

}  // namespace

RSVD_HIDDEN int launch_pack_operands(const float2* c32, long long N, const OperandLayout& L, int precision,
                                     uint16_t* out, cudaStream_t stream) {
  const size_t bytes = (size_t)operand_planes(precision) * (size_t)L.plane_elems * 2;
  if (cudaMemsetAsync(out, 0, bytes, stream) != cudaSuccess) return RSVD_ECUDA;
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
