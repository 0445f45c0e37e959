// Parameters of the tensor-core compression kernel (compress_tc.cu).
#pragma once

#include "rsvd_internal.cuh"

namespace rsvd {

struct CompressTcParams {
  const float2* polar;  // [N][R][Q]
  float2* out;          // [N*T][H][Q/2], FP32 layout of rsvd_compress
  const double* U;      // [R][H]
  int* status;
  int N, R, Q, H, T;
  int uniform;  // rings equispaced: k_r = (r + 1) dk
  float dk;
  float k[kMaxR];
  float sw[kMaxR];
  float dx[kMaxT];
  float dy[kMaxT];
};

// RSVD_EUNSUPPORTED outside Q in {256, 512}, R <= 128, H <= 16.
RSVD_HIDDEN int launch_compress_tc(const CompressTcParams& p, cudaStream_t stream);

}  // namespace rsvd
