// Finer rotation grid by shifted coarse passes (section 2.4, after eq.
// image_innerproduct). The zero-padded landscape at the angles
// gamma_m + 2 pi p / (P Q) (p = 0..P-1) is the coarse landscape of the templates
// rotated by p / P of a grid step:
//   b'_h(q) = b_h(q) e^{-i q 2 pi p / (P Q)} for 0 < |q| < Q/2,  b'_h(0) = b_h(0),
//   b'_h(Q/2) = b_h(Q/2) cos(pi p / P)
// (the Nyquist coefficient is shared by +-Q/2 in the interpolant, and
// X_hat(Q/2) cos(Q gamma / 2) = (-1)^m X_hat(Q/2) cos(pi p / P) at those angles).
// So P passes of the fused scoring kernel (rsvd_align_best) against the
// shifted template rings, merged in place, give max / argmax / log-sum-exp
// over the P Q angles.
#include "operand.cuh"

namespace rsvd {
namespace {

// FP32 packed half spectrum [N_B][H][M]: slot 0 = (Re b(0), Re b(Q/2)), slot s = b(s)
__global__ void shift_templates_kernel(const float2* __restrict__ cB, float2* __restrict__ out, long long n,
                                       int M, int P, int p) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = (int)(i % M);
  const float2 v = cB[i];
  if (s == 0) {
    out[i] = make_float2(v.x, v.y * cospif((float)p / (float)P));
  } else {
    float sn, cs;
    sincospif(-(float)(p * s) / (float)(P * M), &sn, &cs);
    out[i] = make_float2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
  }
}

// pass p into the running result: arg of pass p is t Q + m -> fine index
// t P Q + P m + p; ties keep the smaller fine index; lse combined by log-sum-exp
__global__ void fine_merge_kernel(const float* __restrict__ bp, const int32_t* __restrict__ ap,
                                  const float* __restrict__ lp, long long n, int Q, int P, int p, float* best,
                                  int32_t* arg, float* lse) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = ap[i];
  const int fi = (a / Q) * P * Q + P * (a % Q) + p;
  const float v = bp[i];
  if (p == 0) {
    best[i] = v;
    arg[i] = fi;
    if (lse) lse[i] = lp[i];
    return;
  }
  const float bv = best[i];
  if (v > bv || (v == bv && fi < arg[i])) {
    best[i] = v;
    arg[i] = fi;
  }
  if (lse) {
    const float x = lse[i], y = lp[i];
    const float m = fmaxf(x, y);
    lse[i] = m == -INFINITY ? m : m + logf(expf(x - m) + expf(y - m));
  }
}

struct FineLayout {
  size_t tmpl, best, arg, lse, total;
};

FineLayout fine_layout(int N_A, int N_B, int H, int Q, bool want_lse) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  FineLayout L{};
  L.tmpl = up((size_t)N_B * H * (Q / 2) * sizeof(float2));
  const size_t n = (size_t)N_A * N_B;
  L.best = up(n * sizeof(float));
  L.arg = up(n * sizeof(int32_t));
  L.lse = want_lse ? up(n * sizeof(float)) : 0;
  L.total = L.tmpl + L.best + L.arg + L.lse;
  return L;
}

}  // namespace
}  // namespace rsvd

extern "C" size_t rsvd_align_fine_workspace_bytes(int N_A, int N_B, int H, int Q, int P, int want_lse) {
  if (N_A <= 0 || N_B <= 0 || H <= 0 || Q <= 0 || P < 1) return 0;
  return rsvd::fine_layout(N_A, N_B, H, Q, want_lse != 0).total;
}

extern "C" int rsvd_align_best_fine_shifted(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                            int P, float inv_sigma2, float* best, int32_t* arg, float* lse,
                                            void* workspace, size_t workspace_bytes, void* stream) {
  using namespace rsvd;
  if (!cA || !cB || !best || !arg || N_A <= 0 || N_B <= 0 || T <= 0 || H <= 0) return RSVD_EINVAL;
  if (P < 1 || P > 8 || (P & (P - 1)) || Q < 16 || (Q & (Q - 1))) return RSVD_EUNSUPPORTED;
  if ((long long)T * P * Q > 0x7fffffffLL / 2) return RSVD_EUNSUPPORTED;
  const bool want_lse = lse != nullptr;
  const FineLayout L = fine_layout(N_A, N_B, H, Q, want_lse);
  if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return RSVD_EWORKSPACE;
  char* ws = static_cast<char*>(workspace);
  float2* tshift = reinterpret_cast<float2*>(ws);
  float* bp = reinterpret_cast<float*>(ws + L.tmpl);
  int32_t* ap = reinterpret_cast<int32_t*>(ws + L.tmpl + L.best);
  float* lp = want_lse ? reinterpret_cast<float*>(ws + L.tmpl + L.best + L.arg) : nullptr;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long nt = (long long)N_B * H * (Q / 2), n = (long long)N_A * N_B;
  for (int p = 0; p < P; ++p) {
    const void* tb = cB;
    if (p > 0) {
      shift_templates_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(static_cast<const float2*>(cB), tshift,
                                                                           nt, Q / 2, P, p);
      int rc = launch_status();
      if (rc != RSVD_OK) return rc;
      tb = tshift;
    }
    int rc = rsvd_align_best(cA, N_A, T, tb, N_B, H, Q, RSVD_FP32, inv_sigma2, bp, ap, lp, stream);
    if (rc != RSVD_OK) return rc;
    fine_merge_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(bp, ap, lp, n, Q, P, p, best, arg, lse);
    if ((rc = launch_status()) != RSVD_OK) return rc;
  }
  return RSVD_OK;
}
