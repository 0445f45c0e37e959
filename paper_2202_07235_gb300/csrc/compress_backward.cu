// rsvd_compress_backward: adjoint of rsvd_compress (U held fixed).
//
// Given the gradient with respect to the compressed rings, G_c(row, h, q) for
// q = 0..Q/2 in the packed slot layout (slot 0 = the real q = 0 and q = Q/2
// terms), returns the gradient with respect to the polar samples in the
// convention G = dL/dRe + i dL/dIm, reversing the forward steps of section 3.2
// and eq. image_innerproduct_pm with the translation of section 5:
//   G_c(h, Q-q)   = (-1)^q conj(G_c(h, q))          (pairing of real images)
//   G_a(h, psi)   = (1/Q) sum_{q<Q} e^{+2 pi i q psi / Q} G_c(h, q)
//   G_F(r, psi)   = sum_t exp(+i k_r (dx_t cos psi + dy_t sin psi)) sum_h U_rh sqrt(w_r) G_a,t(h, psi)
// for psi < Q/2; the other half is the conjugate, G_F(r, psi + pi) = conj(G_F(r, psi)).
//
// One CTA per object; translations and principal vectors are processed in
// chunks whose spectra fit in shared memory; the CTA accumulates into its own
// rows of the output (no atomics).
#include <math.h>

#include "rsvd_internal.cuh"

namespace rsvd {
namespace {

constexpr int kThreads = 256;

struct CompressBwdParams {
  const float2* gC;  // [N*T][H][Q/2]
  float2* gpolar;    // [N][R][Q]
  const double* U;   // [R][H]
  int N, R, Q, H, T, TC, HC, log2Q;
  float k[kMaxR];
  float sw[kMaxR];
  float dx[kMaxT];
  float dy[kMaxT];
};

__device__ __forceinline__ int bitrev_n(int i, int bits) { return (int)(__brev((unsigned)i) >> (32 - bits)); }

__global__ void __launch_bounds__(kThreads) compress_bwd_kernel(const __grid_constant__ CompressBwdParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Q = p.Q, M = Q / 2, R = p.R, H = p.H, T = p.T, TC = p.TC, HC = p.HC;
  float* W = reinterpret_cast<float*>(smem_raw);                   // [R][HC] of the current h chunk
  float2* tw = reinterpret_cast<float2*>(W + ((R * HC + 3) & ~3));  // [M] e^{+2 pi i k / Q}
  float2* buf = tw + M;                                            // [TC][HC][Q]
  const int n = blockIdx.x, tid = threadIdx.x;
  if (n >= p.N) return;
  for (int i = tid; i < M; i += kThreads) {
    float sn, cs;
    sincospif(2.0f * (float)i / (float)Q, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
  const float invQ = 1.0f / (float)Q;
  const int nseq = TC * HC;
  float2* out = p.gpolar + (size_t)n * R * Q;

  for (int t0 = 0; t0 < T; t0 += TC) {
    for (int h0 = 0; h0 < H; h0 += HC) {
      const bool first = (t0 == 0 && h0 == 0);
      const bool last = (t0 + TC >= T) && (h0 + HC >= H);
      __syncthreads();  // previous chunk's readers of W / buf are done
      for (int i = tid; i < R * HC; i += kThreads) {
        const int r = i / HC, hh = i % HC;
        const int h = h0 + hh;
        W[i] = (h < H) ? (float)p.U[r * H + h] * p.sw[r] : 0.0f;
      }
      // full spectra in bit-reversed order
      for (int i = tid; i < nseq * Q; i += kThreads) {
        const int seq = i / Q, q = i % Q;
        const int tc = seq / HC, hh = seq % HC;
        const int t = t0 + tc, h = h0 + hh;
        float2 v = make_float2(0.f, 0.f);
        if (t < T && h < H) {
          const float2* g = p.gC + (((size_t)n * T + t) * H + h) * M;
          if (q == 0) {
            v = make_float2(g[0].x, 0.f);
          } else if (q == M) {
            v = make_float2(g[0].y, 0.f);
          } else if (q < M) {
            v = g[q];
          } else {
            const float2 u = g[Q - q];
            v = (q & 1) ? make_float2(-u.x, u.y) : make_float2(u.x, -u.y);  // (-1)^q conj
          }
        }
        buf[(size_t)seq * Q + bitrev_n(q, p.log2Q)] = v;
      }
      __syncthreads();
      // inverse FFTs (e^{+}), radix 2
      for (int half = 1; half < Q; half *= 2) {
        const int stride = M / half;
        for (int bfly = tid; bfly < nseq * M; bfly += kThreads) {
          const int seq = bfly / M, j = bfly % M;
          const int pos = j % half, grp = j / half;
          float2* x = buf + (size_t)seq * Q;
          const int i0 = grp * 2 * half + pos, i1 = i0 + half;
          const float2 a = x[i0];
          const float2 bw = cmul(x[i1], tw[pos * stride]);
          x[i0] = cadd(a, bw);
          x[i1] = csub(a, bw);
        }
        __syncthreads();
      }
      // back-projection, conjugate phase, sum over the translations of the chunk
      for (int i = tid; i < M * R; i += kThreads) {
        const int psi = i % M, r = i / M;
        float sp, cp;
        sincospif(2.0f * (float)psi / (float)Q, &sp, &cp);
        float2 acc = make_float2(0.f, 0.f);
        for (int tc = 0; tc < TC && t0 + tc < T; ++tc) {
          const int t = t0 + tc;
          float gx = 0.f, gy = 0.f;
          for (int hh = 0; hh < HC; ++hh) {
            const float wv = W[r * HC + hh];
            const float2 v = buf[((size_t)tc * HC + hh) * Q + psi];
            gx = fmaf(wv, v.x, gx);
            gy = fmaf(wv, v.y, gy);
          }
          float s, c;
          sincosf(p.k[r] * (p.dx[t] * cp + p.dy[t] * sp), &s, &c);
          // (gx + i gy) * exp(+i theta)
          acc.x += c * gx - s * gy;
          acc.y += c * gy + s * gx;
        }
        acc.x *= invQ;
        acc.y *= invQ;
        float2* o = out + (size_t)r * Q + psi;
        if (!first) {
          const float2 prev = *o;
          acc.x += prev.x;
          acc.y += prev.y;
        }
        *o = acc;
        if (last) o[M] = make_float2(acc.x, -acc.y);
      }
    }
  }
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_compress_backward(int R, int Q, const double* k, const double* w, const double* U, int H,
                                      const void* gC, int N, const double* deltas, int T, int precision, void* gpolar,
                                      void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!k || !w || !U || !gC || !gpolar || N <= 0) return RSVD_EINVAL;
  if (deltas == nullptr) {
    if (T != 1) return RSVD_EINVAL;
  } else if (T <= 0) {
    return RSVD_EINVAL;
  }
  if (T > kMaxT) return RSVD_EUNSUPPORTED;
  if (precision != RSVD_FP32) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)gC & 7u) || ((uintptr_t)gpolar & 7u) || ((uintptr_t)U & 7u)) return RSVD_EINVAL;
  CompressBwdParams p{};
  p.gC = static_cast<const float2*>(gC);
  p.gpolar = static_cast<float2*>(gpolar);
  p.U = U;
  p.N = N;
  p.R = R;
  p.Q = Q;
  p.H = H;
  p.T = T;
  // spectra of TC translations x HC vectors of length Q in at most 96 KB
  const int cap = (96 * 1024) / (Q * 8);
  p.HC = H < cap ? H : (cap > 0 ? cap : 1);
  int tc = cap / p.HC;
  tc = tc < 1 ? 1 : tc;
  p.TC = tc < T ? tc : T;
  int lg = 0;
  while ((1 << lg) < Q) ++lg;
  p.log2Q = lg;
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    p.k[r] = (float)k[r];
    p.sw[r] = (float)sqrt(w[r]);
  }
  for (int t = 0; t < T; ++t) {
    p.dx[t] = deltas ? (float)deltas[2 * t] : 0.0f;
    p.dy[t] = deltas ? (float)deltas[2 * t + 1] : 0.0f;
  }
  const size_t smem = (size_t)((R * p.HC + 3) & ~3) * sizeof(float) + (size_t)(Q / 2) * sizeof(float2) +
                      (size_t)p.TC * p.HC * Q * sizeof(float2);
  if (smem > 227 * 1024) return RSVD_EUNSUPPORTED;
  if (cudaFuncSetAttribute(compress_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RSVD_ECUDA;
  compress_bwd_kernel<<<N, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  return launch_status();
}
