// rsvd_compress: translated principal-image-rings in the Fourier-Bessel basis.
//
// Paper section 3.2 (principal-image-rings [u^T A](psi_q) = sum_r u_r A(k_r, psi_q) eta_r,
// here with eta_r -> sqrt(w_r)), eq. (image_innerproduct_pm) (Fourier-Bessel
// coefficients of the compressed rings, section 2.3 discrete definition) and
// the translation operator T_delta of section 5 ((T_delta A)^ = A^ exp(-i k.delta)).
//
// One CTA per object. For each translation t and block of 16 principal
// vectors h:
//   phase A  thread per angle psi < Q/2:  a_t(h, psi) = sum_r W[r][h] A(r, psi) phi_t(r, psi),
//            W = U * sqrt(w), phi_t = exp(-i k_r (dx cos psi + dy sin psi)); the
//            second half of the ring follows from a(h, psi + pi) = conj(a(h, psi))
//            (real images), so only half of each input ring is read;
//   phase B  Q-point FFT over psi in shared memory (radix-2, bit-reversed input);
//   write    slots s = 0 .. Q/2-1 of a_t(h, q) / Q, slot 0 packing (Re a(0), Re a(Q/2)).
#include <math.h>

#include "compress_tc.cuh"
#include "compress_v2.cuh"
#include "operand.cuh"

namespace rsvd {
namespace {

constexpr int kThreads = 256;
constexpr int kHB = 16;  // principal vectors per register block

struct CompressParams {
  const float2* polar;  // [N][R][Q]
  float2* out;          // [N*T][H][Q/2] (RSVD_FP32)
  uint16_t* planes;     // operand planes (other precisions; layout L)
  OperandLayout L;
  const double* U;      // [R][H]
  int* status;
  int N, R, Q, H, T, Hpad, log2Q, precision;
  float k[kMaxR];
  float sw[kMaxR];
  float dx[kMaxT];
  float dy[kMaxT];
};

__device__ __forceinline__ int bitrev(int i, int bits) { return (int)(__brev((unsigned)i) >> (32 - bits)); }

__global__ void __launch_bounds__(kThreads) compress_kernel(const __grid_constant__ CompressParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Q = p.Q, M = Q / 2, R = p.R, H = p.H, T = p.T, Hpad = p.Hpad;
  const int L = M < kThreads ? M : kThreads;  // threads per translation
  const int CT = kThreads / L;                // translations processed together
  float* W = reinterpret_cast<float*>(smem_raw);                       // [R][Hpad]
  float2* tw = reinterpret_cast<float2*>(W + ((R * Hpad + 3) & ~3));  // [M]  W_Q^k
  float2* buf = tw + M;                                                // [CT][kHB][Q]

  const int n = blockIdx.x;
  const int tid = threadIdx.x;
  if (n >= p.N) return;

  for (int i = tid; i < R * Hpad; i += kThreads) {
    const int r = i / Hpad, h = i % Hpad;
    W[i] = (h < H) ? (float)(p.U[r * H + h]) * p.sw[r] : 0.0f;
  }
  for (int i = tid; i < M; i += kThreads) {
    float s, c;
    sincospif(-2.0f * (float)i / (float)Q, &s, &c);
    tw[i] = make_float2(c, s);
  }
  __syncthreads();

  const int tgrp = tid / L, lane = tid % L;
  const float2* img = p.polar + (size_t)n * R * Q;
  const float invQ = 1.0f / (float)Q;

  for (int t0 = 0; t0 < T; t0 += CT) {
    const int t = t0 + tgrp;
    const bool t_ok = (t < T);
    for (int h0 = 0; h0 < Hpad; h0 += kHB) {
      // ---- phase A: translate + project, half ring per thread-lane ----
      for (int psi = lane; psi < M; psi += L) {
        float acc_re[kHB], acc_im[kHB];
#pragma unroll
        for (int hh = 0; hh < kHB; ++hh) acc_re[hh] = acc_im[hh] = 0.0f;
        if (t_ok) {
          float sp, cp;
          sincospif(2.0f * (float)psi / (float)Q, &sp, &cp);
          const float rho = p.dx[t] * cp + p.dy[t] * sp;
          for (int r = 0; r < R; ++r) {
            const float2 a = img[(size_t)r * Q + psi];
            float s, c;
            sincosf(p.k[r] * rho, &s, &c);
            // a * exp(-i theta)
            const float vr = fmaf(a.x, c, a.y * s);
            const float vi = fmaf(a.y, c, -a.x * s);
            const float* wr = W + r * Hpad + h0;
#pragma unroll
            for (int hh = 0; hh < kHB; ++hh) {
              acc_re[hh] = fmaf(wr[hh], vr, acc_re[hh]);
              acc_im[hh] = fmaf(wr[hh], vi, acc_im[hh]);
            }
          }
        }
        float2* b = buf + (size_t)tgrp * kHB * Q;
        const int i0 = bitrev(psi, p.log2Q), i1 = bitrev(psi + M, p.log2Q);
#pragma unroll
        for (int hh = 0; hh < kHB; ++hh) {
          b[hh * Q + i0] = make_float2(acc_re[hh], acc_im[hh]);
          b[hh * Q + i1] = make_float2(acc_re[hh], -acc_im[hh]);
        }
      }
      __syncthreads();
      // ---- phase B: CT*kHB FFTs of length Q (forward, e^{-i}) ----
      const int nseq = CT * kHB;
      for (int half = 1; half < Q; half *= 2) {
        const int stride = M / half;  // twiddle index step
        for (int bfly = tid; bfly < nseq * M; bfly += kThreads) {
          const int seq = bfly / M, j = bfly % M;
          const int pos = j % half, grp = j / half;
          float2* x = buf + (size_t)seq * Q;
          const int i0 = grp * 2 * half + pos, i1 = i0 + half;
          const float2 w = tw[pos * stride];
          const float2 a = x[i0];
          const float2 bw = cmul(x[i1], w);
          x[i0] = cadd(a, bw);
          x[i1] = csub(a, bw);
        }
        __syncthreads();
      }
      // ---- write slots ----
      for (int i = tid; i < nseq * M; i += kThreads) {
        const int seq = i / M, s = i % M;
        const int tg = seq / kHB, hh = seq % kHB;
        const int tt = t0 + tg, h = h0 + hh;
        if (tt < T && h < H) {
          const float2* x = buf + (size_t)seq * Q;
          float2 v = (s == 0) ? make_float2(x[0].x, x[M].x) : x[s];
          v.x *= invQ;
          v.y *= invQ;
          if (p.precision == RSVD_FP32) {
            const size_t row = (size_t)n * T + tt;
            p.out[(row * H + h) * M + s] = v;
          } else {
            operand_put(p.planes, p.L.plane_elems, p.precision, operand_index(p.L, n, tt, h, s), v);
          }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_compress(int R, int Q, const double* k, const double* w, const double* U, int H,
                             const void* polar, int N, const double* deltas, int T, int precision,
                             void* out, void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!k || !w || !U || !polar || !out || N <= 0) return RSVD_EINVAL;
  if (deltas == nullptr) {
    if (T != 1) return RSVD_EINVAL;
  } else if (T <= 0) {
    return RSVD_EINVAL;
  }
  if (T > kMaxT) return RSVD_EUNSUPPORTED;
  OperandLayout OL{};
  const bool fits_v2 = R * (Q / 2) * 8 <= 96 * 1024;
  if (precision != RSVD_FP32) {
    if (!is_operand_precision(precision)) return RSVD_EUNSUPPORTED;
    if (!make_operand_layout(N, T, H, Q, &OL)) return RSVD_EUNSUPPORTED;
  }
  if (((uintptr_t)polar & 7u) || ((uintptr_t)out & 15u) || ((uintptr_t)U & 7u)) return RSVD_EINVAL;
  if ((size_t)N * T > (size_t)INT32_MAX / 2) return RSVD_EUNSUPPORTED;
  if (precision == RSVD_FP16X3) {
    // the row scaling needs each row's largest component before any part is
    // rounded: FP32 rings into a stream-ordered temporary, then the scaled pack
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* tmp = nullptr;
    if (cudaMallocAsync(&tmp, (size_t)N * T * H * (Q / 2) * 8, st) != cudaSuccess) return RSVD_ECUDA;
    int rc32 = rsvd_compress(R, Q, k, w, U, H, polar, N, deltas, T, RSVD_FP32, tmp, stream);
    if (rc32 == RSVD_OK)
      rc32 = launch_pack_operands(static_cast<const float2*>(tmp), N, OL, RSVD_FP16X3, static_cast<uint16_t*>(out), st);
    const cudaError_t fe = cudaFreeAsync(tmp, st);
    return (rc32 == RSVD_OK && fe != cudaSuccess) ? RSVD_ECUDA : rc32;
  }

  CompressParams p{};
  p.polar = static_cast<const float2*>(polar);
  p.out = static_cast<float2*>(out);
  p.U = U;
  p.status = status_word();
  p.N = N;
  p.R = R;
  p.Q = Q;
  p.H = H;
  p.T = T;
  p.precision = precision;
  p.planes = static_cast<uint16_t*>(out);
  p.L = OL;
  p.Hpad = (H + kHB - 1) / kHB * kHB;
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
  if (precision != RSVD_FP32) {
    // padding components, lanes and tiles of the operand planes are zero
    const size_t bytes = (size_t)operand_planes(precision) * (size_t)OL.plane_elems * 2;
    if (cudaMemsetAsync(out, 0, bytes, static_cast<cudaStream_t>(stream)) != cudaSuccess) return RSVD_ECUDA;
  }
  if (precision == RSVD_FP32 && !fits_v2) {
    // projection on the tensor cores (compress_tc.cu): Q in {256, 512}, R <= 128, H <= 16,
    // where the shared-memory kernel cannot hold the rings (it is the faster
    // one where it can: 1.87 ms against 2.9 ms on the throughput workload)
    CompressTcParams c{};
    c.polar = p.polar;
    c.out = p.out;
    c.U = U;
    c.status = p.status;
    c.N = N;
    c.R = R;
    c.Q = Q;
    c.H = H;
    c.T = T;
    bool uniform = k[0] > 0.0;
    for (int r = 0; r < R && uniform; ++r) uniform = fabs(k[r] - (r + 1) * k[0]) <= 1e-9 * k[R - 1];
    c.uniform = uniform ? 1 : 0;
    c.dk = (float)k[0];
    for (int r = 0; r < R; ++r) {
      c.k[r] = p.k[r];
      c.sw[r] = p.sw[r];
    }
    for (int t = 0; t < T; ++t) {
      c.dx[t] = p.dx[t];
      c.dy[t] = p.dy[t];
    }
    const int rc_tc = launch_compress_tc(c, static_cast<cudaStream_t>(stream));
    if (rc_tc != RSVD_EUNSUPPORTED) return rc_tc;
  }
  {
    // shared-memory kernel when half of one object's rings fits (compress_v2.cu)
    Compress2Params q{};
    q.polar = p.polar;
    q.out = p.out;
    q.U = U;
    q.N = N;
    q.R = R;
    q.Q = Q;
    q.H = H;
    q.T = T;
    bool uniform = k[0] > 0.0;
    for (int r = 0; r < R && uniform; ++r) uniform = fabs(k[r] - (r + 1) * k[0]) <= 1e-9 * k[R - 1];
    q.uniform = uniform ? 1 : 0;
    q.precision = precision;
    q.planes = static_cast<uint16_t*>(out);
    q.L = OL;

    q.dk = (float)k[0];
    for (int r = 0; r < R; ++r) {
      q.k[r] = p.k[r];
      q.sw[r] = p.sw[r];
    }
    for (int t = 0; t < T; ++t) {
      q.dx[t] = p.dx[t];
      q.dy[t] = p.dy[t];
    }
    const int rc2 = fits_v2 ? launch_compress_v2(q, static_cast<cudaStream_t>(stream)) : RSVD_EUNSUPPORTED;
    if (rc2 != RSVD_EUNSUPPORTED) return rc2;
  }
  const int M = Q / 2;
  const int L = M < kThreads ? M : kThreads;
  const int CT = kThreads / L;
  size_t smem = ((size_t)((R * p.Hpad + 3) & ~3)) * sizeof(float) + (size_t)M * sizeof(float2) +
                (size_t)CT * kHB * Q * sizeof(float2);
  if (smem > 227 * 1024) return RSVD_EUNSUPPORTED;
  if (cudaFuncSetAttribute(compress_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return RSVD_ECUDA;
  compress_kernel<<<N, kThreads, smem, static_cast<cudaStream_t>(stream)>>>(p);
  return launch_status();
}
