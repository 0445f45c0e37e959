// Log-sum-exp loss: per-image normaliser and the gradient with respect to
// the compressed rings (entry points rsvd_lse_rows, rsvd_lse_backward).
#include <math.h>

#include "align_grad.cuh"

namespace rsvd {
namespace {

// L[n] = log sum_j exp(lse[n][j]), one warp per image.
__global__ void lse_rows_kernel(const float* __restrict__ lse, int N_A, int N_B, float* __restrict__ L) {
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x % 32;
  if (warp >= N_A) return;
  float m = -INFINITY, s = 0.f;
  for (int j = lane; j < N_B; j += 32) lse_merge(m, s, lse[warp * N_B + j], 1.0f);
  lse_warp_reduce(m, s, 32);
  if (lane == 0) L[warp] = m + logf(s);
}

// out[i] = sum_k partial[k][i] (fixed order: deterministic); with `accumulate`
// the sum is added to out[i].
__global__ void sum_splits_kernel(const float2* __restrict__ partial, int nsplit, size_t n, float2* __restrict__ out,
                                  int accumulate) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float2 acc = partial[i];
    for (int k = 1; k < nsplit; ++k) {
      const float2 v = partial[(size_t)k * n + i];
      acc.x += v.x;
      acc.y += v.y;
    }
    if (accumulate) {
      const float2 o = out[i];
      acc.x += o.x;
      acc.y += o.y;
    }
    out[i] = acc;
  }
}

int padded_h_grad(int H) {
  const int opts[] = {8, 12, 16, 24, 32};
  for (int v : opts)
    if (H <= v) return v;
  return -1;
}

int tmpl_rows(int Q, int HP) {
  if (Q == 128) return grad_tmpl_rows<64>(HP);
  if (Q == 256) return grad_tmpl_rows<128>(HP);
  if (Q == 512) return grad_tmpl_rows<256>(HP);
  return 0;
}

// SMs of the current device (152 on GB300 when the query is unavailable, e.g.
// a size query on a host without a GPU; the launch and its workspace query
// then agree as long as they run on the same device).
int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0) {
    (void)cudaGetLastError();
    return 152;
  }
  return sms;
}

// Splits of the image rows for the template gradient (one CTA per split and
// group of resident templates, one CTA per SM): at least enough CTAs to fill
// the GPU twice, each split at least 64 rows, and among up to four times that
// many splits the first whose CTAs fill their last wave to 95 % (else the
// fullest): 64 groups x 5 splits on 152 SMs left the third wave 11 % full.
int choose_splits(int rows, int N_B, int Q, int HP) {
  const int rp = tmpl_rows(Q, HP);
  if (rp <= 0) return 0;
  const int sms = device_sms();
  const long long groups = (N_B + rp - 1) / rp;
  const int cap = rows / 64 > 1 ? rows / 64 : 1;
  int ns0 = (int)((2LL * sms + groups - 1) / groups);
  ns0 = ns0 < 1 ? 1 : (ns0 < cap ? ns0 : cap);
  int best = ns0;
  double best_fill = 0.0;
  for (int ns = ns0; ns <= 4 * ns0 && ns <= cap; ++ns) {
    const long long ctas = groups * ns, waves = (ctas + sms - 1) / sms;
    const double fill = (double)ctas / (double)(waves * sms);
    if (fill > best_fill + 1e-9) {
      best = ns;
      best_fill = fill;
    }
    if (fill >= 0.95) break;
  }
  return best;
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_lse_rows(const float* lse, int N_A, int N_B, float* L, void* stream) {
  using namespace rsvd;
  if (!lse || !L || N_A <= 0 || N_B <= 0) return RSVD_EINVAL;
  const long long threads = (long long)N_A * 32;
  const int block = 256;
  const long long grid = (threads + block - 1) / block;
  if (grid > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
  lse_rows_kernel<<<(unsigned)grid, block, 0, static_cast<cudaStream_t>(stream)>>>(lse, N_A, N_B, L);
  return launch_status();
}

extern "C" size_t rsvd_lse_backward_workspace_bytes(int N_A, int T, int N_B, int H, int Q) {
  using namespace rsvd;
  if (N_A <= 0 || T <= 0 || N_B <= 0 || H <= 0 || Q <= 0) return 0;
  const int HP = padded_h_grad(H);
  if (HP < 0) return 0;
  const int ns = choose_splits(N_A * T, N_B, Q, HP);
  if (ns <= 0) return 0;
  return (size_t)ns * N_B * H * (Q / 2) * sizeof(float2);
}

namespace rsvd {
namespace {
int lse_backward(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                 float inv_sigma2, const float* L, const float* gL, void* gA, void* gB, void* workspace,
                 size_t workspace_bytes, int accumulate, void* stream) {
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if (!L || !gL || !gA || !gB) return RSVD_EINVAL;
  if (!(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
  if (((uintptr_t)gA & 15u) || ((uintptr_t)gB & 15u)) return RSVD_EINVAL;
  const int HP = padded_h_grad(H);
  if (HP < 0 || (Q != 128 && Q != 256 && Q != 512)) return RSVD_EUNSUPPORTED;
  const int rows = N_A * T;
  const int ns = choose_splits(rows, N_B, Q, HP);
  const size_t need = (size_t)ns * N_B * H * (Q / 2) * sizeof(float2);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 15u)) return RSVD_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  auto launch = [&](bool tmpl, const GradParams& gp) {
    if (Q == 128) return launch_grad_s64(HP, tmpl, gp, st);
    if (Q == 256) return launch_grad_s128(HP, tmpl, gp, st);
    return launch_grad_s256(HP, tmpl, gp, st);
  };
  GradParams pa{};
  pa.res = static_cast<const float2*>(cA);
  pa.str = static_cast<const float2*>(cB);
  pa.out = static_cast<float2*>(gA);
  pa.L = L;
  pa.gL = gL;
  pa.status = status_word();
  pa.H = H;
  pa.T = T;
  pa.n_res = rows;
  pa.n_str = N_B;
  pa.nsplit = 1;
  pa.inv_sigma2 = inv_sigma2;
  if ((rc = launch(false, pa)) != RSVD_OK) return rc;

  GradParams pb = pa;
  pb.res = static_cast<const float2*>(cB);
  pb.str = static_cast<const float2*>(cA);
  pb.out = static_cast<float2*>(workspace);
  pb.n_res = N_B;
  pb.n_str = rows;
  pb.nsplit = ns;
  if ((rc = launch(true, pb)) != RSVD_OK) return rc;

  const size_t n = (size_t)N_B * H * (Q / 2);
  sum_splits_kernel<<<(unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096), 256, 0, st>>>(
      static_cast<const float2*>(workspace), ns, n, static_cast<float2*>(gB), accumulate);
  return launch_status();
}
}  // namespace
}  // namespace rsvd

extern "C" int rsvd_lse_backward(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                                 float inv_sigma2, const float* L, const float* gL, void* gA, void* gB, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  return rsvd::lse_backward(cA, N_A, T, cB, N_B, H, Q, precision, inv_sigma2, L, gL, gA, gB, workspace,
                            workspace_bytes, 0, stream);
}

extern "C" int rsvd_lse_backward_accumulate(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                            int precision, float inv_sigma2, const float* L, const float* gL, void* gA,
                                            void* gB, void* workspace, size_t workspace_bytes, void* stream) {
  return rsvd::lse_backward(cA, N_A, T, cB, N_B, H, Q, precision, inv_sigma2, L, gL, gA, gB, workspace,
                            workspace_bytes, 1, stream);
}
