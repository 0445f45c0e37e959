// Fused scoring kernel for rsvd_align_best (FP32, CUDA cores).
//
// Computes, for every image n, translation t, template j (paper eq.
// image_innerproduct_pm; section 2.7 argmax; section 2.6 likelihood):
//   Step 1  X_hat(q) = 2 pi sum_h conj(a_{n,t}(h, q)) b_j(h, q),  q = 0..Q/2
//   Step 2  X(gamma_m) = sum_{q<Q} e^{-2 pi i q m / Q} X_hat(q)
//   reduce  best/arg = max/argmax over (t, m), lse = log sum_{t,m} exp(s X)
// without writing X (or X_hat) to global memory.
//
// Work decomposition (one CTA per group of IMG images, all their T rows):
// * Thread (g, s) owns angular slot s and keeps RT compressed image rows
//   a(row, 0..H-1, s) in registers for a whole pass; the CTA holds RP = G*RT
//   rows per pass.
// * Templates stream through a double-buffered shared-memory tile of TB
//   templates (cp.async, 16-byte chunks). Each template is read from L2 once per
//   pass and reused by all RP rows.
// * Step 1 for a (row, template) pair is a length-H complex dot product at
//   slot s; the CTA writes the whole half spectrum of RP*TB pairs to shared memory.
// * Step 2 for one pair runs on F = P2 lanes: Q/2 = P1*P2 and lane t takes
//   Z(t + P2 s'), s' < P1 (the C2R pre-processing), does a P1-point DFT in
//   registers, multiplies by W_{Q/2}^{t k1}, exchanges through the pair's own
//   shared-memory region (rows padded to P2+1 so the transposed reads are
//   bank-conflict free and every address is a base plus an immediate), and
//   finishes with P1/P2 P2-point DFTs. Lane outputs z(p) = X(gamma_2p) +
//   i X(gamma_2p+1) are scanned in increasing m for the max/argmax; the
//   log-sum-exp is a second pass of exp2 relative to the pair maximum.
// * Rows of the same image are merged in the CTA (deferred to the next
//   batch's iteration, so each batch costs two barriers); images that span
//   passes are merged through the output arrays (the CTA owns its images, so
//   no atomics are needed and results are deterministic).
#pragma once

#include "align_common.cuh"

namespace rsvd {

struct FusedParams {
  const float2* cA;  // [N_A*T][H][S]
  const float2* cB;  // [N_B][H][S]
  float* best;
  int32_t* arg;
  float* lse;
  int* status;
  int N_A, T, N_B, H, IMG;
  float inv_sigma2;
  // warp-specialised kernel only: CTA b takes image group b % ngroups against
  // templates [c jchunk, (c+1) jchunk), c = b / ngroups (0: all templates)
  int ngroups, jchunk;
};

template <int S>
struct FftSplit;
template <>
struct FftSplit<64> {
  static constexpr int P1 = 8, P2 = 8;
};
template <>
struct FftSplit<128> {
  static constexpr int P1 = 16, P2 = 8;
};
template <>
struct FftSplit<256> {
  static constexpr int P1 = 16, P2 = 16;
};

constexpr int cmin(int a, int b) { return a < b ? a : b; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }
inline int igcd(int a, int b) { return b == 0 ? a : igcd(b, a % b); }
// Images per CTA such that its IMG*T rows fill whole passes of RP rows.
inline int images_per_cta(int RP, int T) { return RP / igcd(RP, T); }

// Pair-region stride (float2): at least the spectrum (S) and the padded
// exchange buffer (P1 rows of P2+1); when a warp holds several pairs (each
// touching 16 banks) consecutive pairs start 16 banks apart.
constexpr int pair_stride(int S, int P1, int P2) {
  const int need = cmax(S, P1 * (P2 + 1));
  return (2 * P2 >= 32) ? (need + 7) / 8 * 8 : ((need - 8 + 15) / 16) * 16 + 8;
}

template <int S, int HP>
struct FusedCfg {
  static constexpr int P1 = FftSplit<S>::P1, P2 = FftSplit<S>::P2;
  static constexpr int RT = cmax(1, cmin(4, 36 / HP));               // image rows per thread
  static constexpr int EST = 2 * RT * HP + 2 * P1 + 2 * P2 + 48;      // register estimate
  static constexpr int G = cmax(1, cmin(cmin(6, 1024 / S), 65536 / (S * EST)));  // row groups
  static constexpr int NT = S * G;                                    // threads
  static constexpr int RP = G * RT;                                   // rows per pass
  static constexpr int XP = P2 + 1;                                   // exchange row stride
  static constexpr int SP = pair_stride(S, P1, P2);                   // pair stride (float2)
  static constexpr int kBudget = 200 * 1024;
  static constexpr int FIXED = 2 * S * 8 + 256;
  static constexpr int PER_TB = 2 * HP * S * 8 + RP * SP * 8 + 2 * RP * 12;
  static constexpr int TB = cmax(1, cmin(16, (kBudget - FIXED) / PER_TB));  // templates per batch
  static constexpr int PAIRS = RP * TB;
  static constexpr size_t SMEM = (size_t)2 * TB * HP * S * 8 + (size_t)PAIRS * SP * 8 + (size_t)2 * S * 8 +
                                 (size_t)2 * PAIRS * 12;
  static constexpr bool kFits = SMEM <= 227 * 1024;
};

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

template <int S, int HP>
__global__ void __launch_bounds__(FusedCfg<S, HP>::NT, 1) fused_align_kernel(const __grid_constant__ FusedParams p) {
  using C = FusedCfg<S, HP>;
  constexpr int M = S, Q = 2 * S, P1 = C::P1, P2 = C::P2, RP = C::RP, RT = C::RT, TB = C::TB, NT = C::NT;
  constexpr int SP = C::SP, XP = C::XP, F = P2, RR = P1 / P2, PAIRS = C::PAIRS, PG = NT / F;
  static_assert(P1 * P2 == M, "FFT split must cover Q/2");
  static_assert(P1 % P2 == 0 && 32 % F == 0, "bad FFT split");

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tbuf = reinterpret_cast<float2*>(smem_raw);  // [2][TB][HP][S], rows h >= H zero
  float2* spec = tbuf + 2 * TB * HP * S;               // [PAIRS][SP]
  float2* twQ = spec + PAIRS * SP;                     // [M]   W_Q^k
  float2* tw1 = twQ + M;                               // [P1][P2]  W_M^{t k1} at k1*P2 + t
  float* res = reinterpret_cast<float*>(tw1 + M);      // [2][3][PAIRS]: best value, argmax m, lse

  const int tid = threadIdx.x;
  const int g = tid / S, s = tid % S;
  const int H = p.H, T = p.T, N_B = p.N_B;
  const int img0 = blockIdx.x * p.IMG;
  if (img0 >= p.N_A) return;
  const int nimg = min(p.IMG, p.N_A - img0);
  const int rows_cta = nimg * T;
  const size_t row0 = (size_t)img0 * T;
  const bool want_lse = (p.lse != nullptr);
  const float s2 = p.inv_sigma2;
  const float two_pi = 6.28318530717958647692f;
  const float log2e = 1.44269504088896340736f;

  for (int i = tid; i < M; i += NT) {
    float sn, cs;
    sincospif(-2.0f * (float)i / (float)Q, &sn, &cs);
    twQ[i] = make_float2(cs, sn);
  }
  for (int i = tid; i < M; i += NT) {
    const int k1 = i / P2, t = i % P2;
    float sn, cs;
    sincospif(-2.0f * (float)(t * k1) / (float)M, &sn, &cs);
    tw1[i] = make_float2(cs, sn);
  }
  // rows h in [H, HP) of every template slot stay zero (the copies fill h < H)
  for (int i = tid; i < 2 * TB * (HP - H) * S; i += NT) {
    const int slot = i / ((HP - H) * S), rem = i % ((HP - H) * S);
    tbuf[(size_t)slot * HP * S + (size_t)H * S + rem] = make_float2(0.f, 0.f);
  }

  const int nbatch = (N_B + TB - 1) / TB;
  const int tsz2 = H * S / 2;  // 16-byte chunks per template

  auto issue_batch = [&](int b, int buf) {
    const int j0 = b * TB;
    const int nb = min(TB, N_B - j0);
    for (int jj = 0; jj < nb; ++jj) {
      const float2* src = p.cB + (size_t)(j0 + jj) * H * S;
      float2* dst = tbuf + (size_t)(buf * TB + jj) * HP * S;
      for (int i = tid; i < tsz2; i += NT) cp_async16(dst + 2 * i, src + 2 * i);
    }
    cp_async_commit();
  };

  // Merge the per-pair results of batch b (rows of one image combined in t
  // order, then with the output written by an earlier pass).
  auto merge = [&](int ps, int b, const float* rs) {
    const float* rv = rs;
    const int* ri = reinterpret_cast<const int*>(rs + PAIRS);
    const float* rl = rs + 2 * PAIRS;
    const int j0 = b * TB, nb = min(TB, N_B - j0);
    const int il0 = ps / T;
    const int il1 = min(nimg - 1, (ps + RP - 1) / T);
    const int nitems = (il1 - il0 + 1) * nb;
    for (int it = tid; it < nitems; it += NT) {
      const int il = il0 + it / nb, jj = it % nb;
      const int rlo = max(il * T - ps, 0), rhi = min((il + 1) * T - ps, RP);
      float vb = -INFINITY, mm = -INFINITY, sm = 0.f;
      int ib = 0x7fffffff;
      for (int rl_ = rlo; rl_ < rhi; ++rl_) {
        const int pr = rl_ * TB + jj;
        const int t = ps + rl_ - il * T;
        const float v = rv[pr];
        if (v > vb || rl_ == rlo) {  // increasing t: ties keep the earlier index
          vb = v;
          ib = t * Q + ri[pr];
        }
        if (want_lse) lse_merge(mm, sm, rl[pr], 1.0f);
      }
      const size_t o = (size_t)(img0 + il) * N_B + j0 + jj;
      if (il * T < ps) {  // earlier passes already stored smaller t
        const float ov = p.best[o];
        if (!(vb > ov)) {
          vb = ov;
          ib = p.arg[o];
        }
        if (want_lse) lse_merge(mm, sm, p.lse[o], 1.0f);
      }
      p.best[o] = vb;
      p.arg[o] = ib;
      if (want_lse) p.lse[o] = mm + logf(sm);
    }
  };

  const bool slot0 = (s == 0);
  const int ft = tid % F;

  for (int ps = 0; ps < rows_cta; ps += RP) {
    // ---- this pass's image rows (times 2 pi), held in registers ----
    float2 a[RT][HP];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const int lr = ps + g * RT + i;
      const bool valid = lr < rows_cta;
      const float2* src = p.cA + ((row0 + (valid ? lr : 0)) * H) * S + s;
#pragma unroll
      for (int h = 0; h < HP; ++h) {
        const float2 v = (valid && h < H) ? src[(size_t)h * S] : make_float2(0.f, 0.f);
        a[i][h] = make_float2(two_pi * v.x, two_pi * v.y);
      }
    }

    issue_batch(0, 0);
    for (int b = 0; b < nbatch; ++b) {
      const int cur = b & 1;
      if (b + 1 < nbatch) {
        issue_batch(b + 1, cur ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();  // templates of batch b landed; FFT of batch b-1 finished
      if (b > 0) merge(ps, b - 1, res + (cur ^ 1) * 3 * PAIRS);
      const int nb = min(TB, N_B - b * TB);

      // ---- Step 1: half spectrum of RP x nb pairs at slot s ----
      const float2* tb = tbuf + (size_t)cur * TB * HP * S + s;
#pragma unroll 1
      for (int jj = 0; jj < TB; ++jj) {
        if (jj < nb) {
          // (P, Qa) = sum_h (a.x b.x, a.y b.y), (Ra, Sa) = sum_h (a.x b.y, a.y b.x): two packed
          // FP32x2 FMAs per row and h; the swapped template value is shared by the RT rows
          float2 PQ[RT], RS[RT];
#pragma unroll
          for (int i = 0; i < RT; ++i) PQ[i] = RS[i] = make_float2(0.f, 0.f);
          const float2* bp = tb + (size_t)jj * HP * S;
#pragma unroll
          for (int h = 0; h < HP; ++h) {
            const float2 bv = bp[h * S];
            const float2 bs = make_float2(bv.y, bv.x);
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              PQ[i] = __ffma2_rn(a[i][h], bv, PQ[i]);
              RS[i] = __ffma2_rn(a[i][h], bs, RS[i]);
            }
          }
          float P[RT], Qa[RT], Ra[RT], Sa[RT];
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            P[i] = PQ[i].x;
            Qa[i] = PQ[i].y;
            Ra[i] = RS[i].x;
            Sa[i] = RS[i].y;
          }
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            // slot 0 packs the real coefficients of q = 0 and q = Q/2
            const float re = slot0 ? P[i] : P[i] + Qa[i];
            const float im = slot0 ? Qa[i] : Ra[i] - Sa[i];
            spec[((g * RT + i) * TB + jj) * SP + s] = make_float2(re, im);
          }
        }
      }
      __syncthreads();  // spectrum complete; template buffer `cur` free

      // ---- Step 2 + per-pair reduction, F lanes per pair ----
      float* rs = res + cur * 3 * PAIRS;
#pragma unroll 1
      for (int pb = 0; pb < PAIRS; pb += PG) {
        const int pr = pb + tid / F;
        const int rl = pr / TB, jj = pr % TB;
        const bool ok = (pr < PAIRS) && (jj < nb) && (ps + rl < rows_cta);
        float2* sp = spec + (size_t)(pr < PAIRS ? pr : 0) * SP;
        float2 z[P1];
        if (ok) {
#pragma unroll
          for (int q1 = 0; q1 < P1; ++q1) {
            const int k = ft + P2 * q1;
            float2 A, B;
            if (q1 == 0 && ft == 0) {
              const float2 v = sp[0];
              A = make_float2(v.x, 0.f);
              B = make_float2(v.y, 0.f);
            } else {
              A = sp[k];
              B = cconj(sp[M - k]);
            }
            const float2 d = cmul(csub(A, B), twQ[k]);
            z[q1] = make_float2(A.x + B.x - d.y, A.y + B.y + d.x);
          }
          RegDft<P1>::run(z);
#pragma unroll
          for (int k1 = 1; k1 < P1; ++k1) z[k1] = cmul(z[k1], tw1[k1 * P2 + ft]);
        }
        __syncwarp();
        if (ok) {
#pragma unroll
          for (int k1 = 0; k1 < P1; ++k1) sp[k1 * XP + ft] = z[k1];
        }
        __syncwarp();
        float2 y[RR][P2];
        float bv = -INFINITY;
        int bj = 0;
        if (ok) {
#pragma unroll
          for (int i = 0; i < RR; ++i) {
#pragma unroll
            for (int tp = 0; tp < P2; ++tp) y[i][tp] = sp[(ft * RR + i) * XP + tp];
            RegDft<P2>::run(y[i]);
          }
          // outputs in increasing m: m = 2 (ft*RR + i + P1*k2) + e
#pragma unroll
          for (int k2 = 0; k2 < P2; ++k2) {
#pragma unroll
            for (int i = 0; i < RR; ++i) {
              const int j = (k2 * RR + i) * 2;
              if (y[i][k2].x > bv) {
                bv = y[i][k2].x;
                bj = j;
              }
              if (y[i][k2].y > bv) {
                bv = y[i][k2].y;
                bj = j + 1;
              }
            }
          }
        }
        int bm = ok ? 2 * (ft * RR + (bj >> 1) % RR + P1 * ((bj >> 1) / RR)) + (bj & 1) : 0x7fffffff;
        argmax_warp_reduce(bv, bm, F);
        float lsev = 0.f;
        if (want_lse) {
          float sum = 0.f;
          if (ok) {
            const float c = s2 * log2e, off = -c * bv;
#pragma unroll
            for (int i = 0; i < RR; ++i)
#pragma unroll
              for (int k2 = 0; k2 < P2; ++k2)
                sum += exp2f(fmaf(c, y[i][k2].x, off)) + exp2f(fmaf(c, y[i][k2].y, off));
          }
#pragma unroll
          for (int off = F / 2; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off, F);
          lsev = s2 * bv + logf(sum);
        }
        if (ok && ft == 0) {
          rs[pr] = bv;
          reinterpret_cast<int*>(rs + PAIRS)[pr] = bm;
          rs[2 * PAIRS + pr] = lsev;
        }
      }
    }
    __syncthreads();  // last batch's FFT finished
    merge(ps, nbatch - 1, res + ((nbatch - 1) & 1) * 3 * PAIRS);
  }
}

template <int S, int HP>
int launch_fused_cfg(const FusedParams& p0, cudaStream_t stream) {
  using C = FusedCfg<S, HP>;
  if constexpr (!C::kFits) {
    return RSVD_EUNSUPPORTED;
  } else {
    FusedParams p = p0;
    p.IMG = images_per_cta(C::RP, p.T);
    const long long grid = ((long long)p.N_A + p.IMG - 1) / p.IMG;
    if (grid > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
    if (cudaFuncSetAttribute(fused_align_kernel<S, HP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::SMEM) != cudaSuccess)
      return RSVD_ECUDA;
    fused_align_kernel<S, HP><<<(unsigned)grid, C::NT, C::SMEM, stream>>>(p);
    return launch_status();
  }
}

template <int S>
int launch_fused_s(int HP, const FusedParams& p, cudaStream_t stream) {
  switch (HP) {
    case 8: return launch_fused_cfg<S, 8>(p, stream);
    case 12: return launch_fused_cfg<S, 12>(p, stream);
    case 16: return launch_fused_cfg<S, 16>(p, stream);
    case 24: return launch_fused_cfg<S, 24>(p, stream);
    case 32: return launch_fused_cfg<S, 32>(p, stream);
    case 64: return launch_fused_cfg<S, 64>(p, stream);
    default: return RSVD_EUNSUPPORTED;
  }
}

RSVD_HIDDEN int launch_fused_s64(int HP, const FusedParams& p, cudaStream_t stream);
RSVD_HIDDEN int launch_fused_s128(int HP, const FusedParams& p, cudaStream_t stream);
RSVD_HIDDEN int launch_fused_s256(int HP, const FusedParams& p, cudaStream_t stream);

}  // namespace rsvd
