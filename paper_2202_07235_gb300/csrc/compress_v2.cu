// Compression kernel for Q in {128, 256, 512} when half of one object's rings
// fits in shared memory (same contract and arithmetic as compress_kernel:
// section 3.2 principal-image-rings with sqrt(w_r) U, the translation T_delta
// of section 5, and the section 2.3 discrete Fourier-Bessel coefficients).
//
// One CTA per object:
// * the half ring set A(r, psi), psi < Q/2, is staged once in shared memory and
//   reused by every translation (the other half is the conjugate);
// * projection item (t, psi): a_t(h, psi) = sum_r W[r][h] A(r, psi) phi_t(r, psi), one
//   packed FP32x2 FMA per (ring, vector) with the weight splatted in shared
//   memory; phi_t(r, psi) = exp(-i k_r rho_t(psi)) is evaluated with sincosf, or, when
//   the rings are equispaced (k_r = r k_1), by multiplying by exp(-i k_1 rho) from
//   ring to ring and re-anchoring with sincosf every 8 rings;
// * the Q-point FFT of each (t, h) sequence (completed by conjugation) runs on P2
//   lanes: P1-point DFTs in registers, twiddles W_Q^{t k1}, an exchange through
//   padded shared memory, P2-point DFTs; slots q = 0..Q/2 are written as in
//   compress_kernel.
#include <math.h>

#include "compress_v2.cuh"

namespace rsvd {
namespace {

template <int Q>
struct C2Split;
template <>
struct C2Split<128> {
  static constexpr int P1 = 16, P2 = 8;
};
template <>
struct C2Split<256> {
  static constexpr int P1 = 16, P2 = 16;
};
template <>
struct C2Split<512> {
  static constexpr int P1 = 32, P2 = 16;
};

constexpr int kBufBudget = 96 * 1024;

constexpr int imax(int a, int b) { return a > b ? a : b; }

template <int Q, int HB>
struct C2Cfg {
  static constexpr int M = Q / 2, P1 = C2Split<Q>::P1, P2 = C2Split<Q>::P2, XP = P2 + 1, RR = P1 / P2;
  static constexpr int SEQ = imax(Q, P1 * XP);                         // float2 per sequence buffer
  static constexpr int TG = imax(1, kBufBudget / (HB * SEQ * 8));      // translations per group
  // threads: one projection item (translation, angle) each when TG * M allows
  static constexpr int NT = (TG * M) % 384 == 0 ? 384 : 256;
  static size_t smem(int R) {
    return (size_t)R * M * 8 + (size_t)R * HB * 8 + (size_t)Q * 8 + (size_t)TG * HB * SEQ * 8;
  }
};

template <int Q, int HB>
__global__ void __launch_bounds__(C2Cfg<Q, HB>::NT) compress2_kernel(const __grid_constant__ Compress2Params p) {
  using C = C2Cfg<Q, HB>;
  constexpr int kNT = C::NT;
  constexpr int M = C::M, P1 = C::P1, P2 = C::P2, XP = C::XP, RR = C::RR, SEQ = C::SEQ, TG = C::TG;
  static_assert(HB % 2 == 0, "HB must be even");
  extern __shared__ __align__(16) unsigned char c2_smem[];
  const int R = p.R, H = p.H, T = p.T;
  float2* img = reinterpret_cast<float2*>(c2_smem);  // [R][M]
  float2* Wsp = img + (size_t)R * M;                  // [R][HB] (w, w)
  float2* tw2 = Wsp + (size_t)R * HB;                 // [P1][P2] W_Q^{t k1}
  float2* buf = tw2 + Q;                              // [TG][HB][SEQ]
  const int n = blockIdx.x, tid = threadIdx.x;
  if (n >= p.N) return;

  // stage the half rings with asynchronous 16-byte copies (two samples each), all
  // in flight at once; M is even and every ring starts 16-byte aligned when the
  // array does, else plain loads
  const float2* src = p.polar + (size_t)n * R * Q;
  if (((uintptr_t)p.polar & 15u) == 0) {
    for (int i = tid; i < R * M / 2; i += kNT) {
      const int r = (2 * i) / M, psi = (2 * i) % M;
      const unsigned d = (unsigned)__cvta_generic_to_shared(img + 2 * i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + (size_t)r * Q + psi) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  } else {
    for (int i = tid; i < R * M; i += kNT) {
      const int r = i / M, psi = i % M;
      img[i] = src[(size_t)r * Q + psi];
    }
  }
  for (int i = tid; i < P1 * P2; i += kNT) {
    const int k1 = i / P2, t = i % P2;
    float sn, cs;
    sincospif(-2.0f * (float)(t * k1) / (float)Q, &sn, &cs);
    tw2[i] = make_float2(cs, sn);
  }
  const float invQ = 1.0f / (float)Q;

  for (int h0 = 0; h0 < H; h0 += HB) {
    __syncthreads();
    for (int i = tid; i < R * HB; i += kNT) {
      const int r = i / HB, hh = i % HB;
      const float wv = (h0 + hh < H) ? (float)p.U[r * H + h0 + hh] * p.sw[r] : 0.0f;
      Wsp[i] = make_float2(wv, wv);
    }
    __syncthreads();
    for (int t0 = 0; t0 < T; t0 += TG) {
      // ---- projection: items (translation, angle) ----
      for (int item = tid; item < TG * M; item += kNT) {
        const int tl = item / M, psi = item % M;
        const int t = t0 + tl;
        float2 acc[HB];
#pragma unroll
        for (int hh = 0; hh < HB; ++hh) acc[hh] = make_float2(0.f, 0.f);
        if (t < T) {
          float spsi, cpsi;
          sincospif(2.0f * (float)psi / (float)Q, &spsi, &cpsi);
          const float rho = p.dx[t] * cpsi + p.dy[t] * spsi;
          float2 step = make_float2(1.f, 0.f), ph = make_float2(1.f, 0.f);
          if (p.uniform) {
            float s, c;
            sincosf(p.dk * rho, &s, &c);
            step = make_float2(c, -s);
          }
          for (int r = 0; r < R; ++r) {
            if (!p.uniform || (r & 7) == 0) {
              float s, c;
              sincosf(p.k[r] * rho, &s, &c);
              ph = make_float2(c, -s);
            } else {
              ph = cmul(ph, step);
            }
            const float2 u = cmul(img[(size_t)r * M + psi], ph);
            const float4* w4 = reinterpret_cast<const float4*>(Wsp + (size_t)r * HB);
#pragma unroll
            for (int hh = 0; hh < HB / 2; ++hh) {
              const float4 ww = w4[hh];
              acc[2 * hh] = __ffma2_rn(make_float2(ww.x, ww.y), u, acc[2 * hh]);
              acc[2 * hh + 1] = __ffma2_rn(make_float2(ww.z, ww.w), u, acc[2 * hh + 1]);
            }
          }
        }
#pragma unroll
        for (int hh = 0; hh < HB; ++hh) {
          float2* x = buf + ((size_t)tl * HB + hh) * SEQ;
          x[psi] = acc[hh];
          x[psi + M] = cconj(acc[hh]);
        }
      }
      __syncthreads();
      // ---- Q-point FFTs, P2 lanes per sequence ----
      const int nseq = TG * HB;
      for (int base = 0; base < nseq * P2; base += kNT) {
        const int idx = base + tid;
        const int seq = idx / P2, tp = idx % P2;
        const bool valid = seq < nseq;
        const int tl = seq / HB, hh = seq % HB;
        const int t = t0 + tl, h = h0 + hh;
        float2* x = buf + (size_t)(valid ? seq : 0) * SEQ;
        float2 z[P1];
#pragma unroll
        for (int s1 = 0; s1 < P1; ++s1) z[s1] = x[tp + P2 * s1];
        RegDft<P1>::run(z);
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) z[k1] = cmul(z[k1], tw2[k1 * P2 + tp]);
        __syncwarp();
        if (valid) {
#pragma unroll
          for (int k1 = 0; k1 < P1; ++k1) x[k1 * XP + tp] = z[k1];
        }
        __syncwarp();
        if (valid && t < T && h < H && p.precision != RSVD_FP32) {
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            const int k1 = tp * RR + i;
            float2 y[P2];
#pragma unroll
            for (int q2 = 0; q2 < P2; ++q2) y[q2] = x[k1 * XP + q2];
            RegDft<P2>::run(y);
#pragma unroll
            for (int k2 = 0; k2 < P2 / 2; ++k2) {
              const int q = k1 + P1 * k2;
              const float2 v = (q == 0) ? make_float2(y[0].x * invQ, y[P2 / 2].x * invQ)
                                        : make_float2(y[k2].x * invQ, y[k2].y * invQ);
              operand_put(p.planes, p.L.plane_elems, p.precision, operand_index(p.L, n, t, h, q), v);
            }
          }
        } else if (valid && t < T && h < H) {
          float2* o = p.out + (((size_t)n * T + t) * H + h) * M;
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            const int k1 = tp * RR + i;
            float2 y[P2];
#pragma unroll
            for (int q2 = 0; q2 < P2; ++q2) y[q2] = x[k1 * XP + q2];
            RegDft<P2>::run(y);
            // X(k1 + P1 k2); slots q = 1 .. M-1, slot 0 = (Re X(0), Re X(M))
#pragma unroll
            for (int k2 = 0; k2 < P2 / 2; ++k2) {
              const int q = k1 + P1 * k2;
              if (q == 0) {
                o[0] = make_float2(y[0].x * invQ, y[P2 / 2].x * invQ);
              } else {
                o[q] = make_float2(y[k2].x * invQ, y[k2].y * invQ);
              }
            }
          }
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
}

template <int Q>
int launch_q(const Compress2Params& p, cudaStream_t stream) {
  const int H = p.H;
  auto go = [&](auto hb_tag) -> int {
    constexpr int HB = decltype(hb_tag)::value;
    using C = C2Cfg<Q, HB>;
    const size_t smem = C::smem(p.R);
    if (smem > 227 * 1024) return RSVD_EUNSUPPORTED;
    if (cudaFuncSetAttribute(compress2_kernel<Q, HB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return RSVD_ECUDA;
    compress2_kernel<Q, HB><<<p.N, C::NT, smem, stream>>>(p);
    return launch_status();
  };
  if (H <= 4) return go(std::integral_constant<int, 4>{});
  if (H <= 8) return go(std::integral_constant<int, 8>{});
  if (H <= 12) return go(std::integral_constant<int, 12>{});
  return go(std::integral_constant<int, 16>{});
}

}  // namespace

RSVD_HIDDEN int launch_compress_v2(const Compress2Params& p, cudaStream_t stream) {
  switch (p.Q) {
    case 128: return launch_q<128>(p, stream);
    case 256: return launch_q<256>(p, stream);
    case 512: return launch_q<512>(p, stream);
    default: return RSVD_EUNSUPPORTED;
  }
}

}  // namespace rsvd
