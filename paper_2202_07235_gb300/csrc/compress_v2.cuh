// Parameters of the shared-memory compression kernel (compress_v2.cu).
#pragma once

#include <type_traits>

#include "operand.cuh"

namespace rsvd {

struct Compress2Params {
  const float2* polar;  // [N][R][Q]
  float2* out;          // [N*T][H][Q/2]
  const double* U;      // [R][H]
  int N, R, Q, H, T;
  int uniform;  // rings equispaced: k_r = (r + 1) dk
  float dk;
  float k[kMaxR];
  float sw[kMaxR];
  float dx[kMaxT];
  float dy[kMaxT];
  // RSVD_FP32: write `out`; otherwise round into the operand planes `planes`
  // (layout `L`, operand.cuh)
  int precision;
  uint16_t* planes;
  OperandLayout L;
};

// RSVD_EUNSUPPORTED when Q or the shared-memory footprint is outside its range.
RSVD_HIDDEN int launch_compress_v2(const Compress2Params& p, cudaStream_t stream);

}  // namespace rsvd
