// Adjoint of the fused scoring for the log-sum-exp alignment loss
// (rsvd_lse_backward).
//
// Loss (section 2.6 likelihood marginalised over rotations, translations and
// templates): sum_n gL_n L_n with L_n = log sum_{j,t,m} exp(s X(n,t,j,m)).
// With P(m) = s gL_n exp(s X(m) - L_n) = dLoss/dX(m):
//   G(q)     = sum_m P(m) e^{+2 pi i q m / Q}                 (q = 0..Q/2)
//   dLoss/da_h(q) = 2 pi sum_j b_h(q) conj(G(q))               (gradient w.r.t. images)
//   dLoss/db_h(q) = 2 pi sum_{n,t} a_h(q) G(q)                 (gradient w.r.t. templates)
// in the packed half-spectrum layout of the compressed rings (slot 0 holds
// the real q = 0 and q = Q/2 terms). X is recomputed, never stored.
//
// One kernel body serves both gradients. A CTA keeps a "resident" set of
// objects in registers (angular slot s per thread, RT objects per thread)
// and streams the other set through double-buffered shared memory:
// * kTmpl = false: resident = image rows (all T rows of IMG images),
//   streamed = all templates; each CTA owns the gradient of its rows.
// * kTmpl = true: resident = RP templates, streamed = a split of the image
//   rows; each CTA writes a partial template gradient that a second kernel
//   sums over splits (deterministic, no atomics).
// Per (resident, streamed) pair and batch: Step 1 at slot s (as the forward),
// the forward two-stage FFT on P2 lanes, P(m) in registers (packed as
// P(2mu) + i P(2mu+1)), the transposed two-stage inverse FFT, the real-to-half
// spectrum post-processing into G(q), then the gradient contraction at slot s.
#pragma once

#include "align_fused.cuh"
#include "ptx_sync.cuh"

namespace rsvd {

struct GradParams {
  const float2* res;  // resident objects [n_res][H][S]
  const float2* str;  // streamed objects [n_str][H][S]
  float2* out;        // images: [n_res][H][S]; templates: partial [nsplit][n_res][H][S]
  const float* L;     // [N_A] per-image log normaliser
  const float* gL;    // [N_A] upstream gradient dLoss/dL_n
  int* status;
  int H, T, n_res, n_str, res_per_cta, nsplit;
  float inv_sigma2;
};

template <int S, int HP>
struct GradCfg {
  static constexpr int P1 = FftSplit<S>::P1, P2 = FftSplit<S>::P2;
  // rows per thread: at Q = 512 the transforms run on 64 lanes with 4 points
  // each (few registers), which leaves room for more resident rows; every
  // resident row reuses each streamed template (32 KB at H = 16)
  static constexpr int RT = (S == 256) ? cmax(1, cmin(3, 48 / HP)) : cmax(1, cmin(3, 24 / HP));
  static constexpr int EST = 4 * RT * HP + 2 * P1 + 4 * P2 + 64;
  static constexpr int G = cmax(1, cmin(cmin(6, 1024 / S), 65536 / (S * EST)));
  static constexpr int NT = S * G;
  static constexpr int RP = G * RT;
  static constexpr int XP = P2 + 1;
  static constexpr int SP = pair_stride(S, P1, P2);
  static constexpr int kBudget = 216 * 1024;
  static constexpr int FIXED = 2 * S * 8 + 8 * RP + 256;
  static constexpr int PER_TB = 2 * HP * S * 8 + RP * SP * 8 + 8;
  static constexpr int TB = cmax(1, cmin(16, (kBudget - FIXED) / PER_TB));
  static constexpr int PAIRS = RP * TB;
  static constexpr size_t SMEM = (size_t)2 * TB * HP * S * 8 + (size_t)PAIRS * SP * 8 + (size_t)2 * S * 8 +
                                 (size_t)2 * RP * 4 + (size_t)2 * TB * 4;
  static constexpr bool kFits = SMEM <= 227 * 1024;
};

// One radix-4 pass of an M-point Stockham transform (in place in `data`, M / 4
// lanes each holding 4 points; forward e^{-}, or e^{+} when kInv) by the
// 64 threads of named barrier `bar`: the lane's inputs are data[j + (M/4) r]
// (loaded when kLoad, else already in v), twiddled by W_M^{r (j % Ns) M / (4 Ns)}
// (tw = W_M^k table), transformed, and written to
// data[(j / Ns) 4 Ns + j % Ns + r Ns] when kStore (else left in v).
template <int M, bool kInv, bool kLoad, bool kStore>
__device__ __forceinline__ void grad_radix4_pass(float2* data, float2 (&v)[4], int j, int Ns, const float2* tw,
                                                 int bar) {
  constexpr int R4 = M / 4;
  if (kLoad) {
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = data[j + R4 * r];
    named_sync(bar, 64);  // every lane has read before any lane writes (here or in the next pass)
  }
  const int e = (j % Ns) * (R4 / Ns);
#pragma unroll
  for (int r = 1; r < 4; ++r) {
    float2 w = tw[(r * e) & (M - 1)];
    if (kInv) w.y = -w.y;
    v[r] = cmul(v[r], w);
  }
  const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]), a3 = csub(v[1], v[3]);
  const float2 ia3 = make_float2(-a3.y, a3.x);  // i a3
  v[0] = cadd(a0, a2);
  v[2] = csub(a0, a2);
  v[1] = kInv ? cadd(a1, ia3) : csub(a1, ia3);
  v[3] = kInv ? csub(a1, ia3) : cadd(a1, ia3);
  if (kStore) {
    const int d = (j / Ns) * 4 * Ns + j % Ns;
#pragma unroll
    for (int r = 0; r < 4; ++r) data[d + r * Ns] = v[r];
    named_sync(bar, 64);  // the pass is visible before the next one reads
  }
}

template <int S, int HP, bool kTmpl>
__global__ void __launch_bounds__(GradCfg<S, HP>::NT, 1) grad_kernel(const __grid_constant__ GradParams p) {
  using C = GradCfg<S, HP>;
  constexpr int M = S, Q = 2 * S, P1 = C::P1, P2 = C::P2, RP = C::RP, RT = C::RT, TB = C::TB, NT = C::NT;
  constexpr int SP = C::SP, XP = C::XP, F = P2, RR = P1 / P2, PAIRS = C::PAIRS, PG = NT / F;
  // Q = 512: each pair's transforms run on 64 lanes (radix-4 Stockham passes),
  // since a batch holds only RP x TB = 3 pairs there
  constexpr bool kWideFft = (S == 256) && (NT % 64 == 0);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tbuf = reinterpret_cast<float2*>(smem_raw);  // [2][TB][HP][S] streamed objects, rows h >= H zero
  float2* spec = tbuf + 2 * TB * HP * S;               // [PAIRS][SP]
  float2* twQ = spec + PAIRS * SP;                     // [M]  W_Q^k
  float2* tw1 = twQ + M;                               // [P1][P2] W_M^{t k1}
  float* rL = reinterpret_cast<float*>(tw1 + M);       // [RP] L of the resident rows' images
  float* rG = rL + RP;                                 // [RP] gL of the resident rows' images
  float* sL = rG + RP;                                 // [TB] L of the streamed rows' images
  float* sG = sL + TB;                                 // [TB]

  const int tid = threadIdx.x;
  const int g = tid / S, s = tid % S;
  const int H = p.H, T = p.T;
  const int res0 = blockIdx.x * p.res_per_cta;
  if (res0 >= p.n_res) return;
  const int nres = min(p.res_per_cta, p.n_res - res0);
  const int split = kTmpl ? blockIdx.y : 0;
  const int str0 = kTmpl ? (int)((long long)p.n_str * split / p.nsplit) : 0;
  const int str1 = kTmpl ? (int)((long long)p.n_str * (split + 1) / p.nsplit) : p.n_str;
  const float s2 = p.inv_sigma2;
  const float two_pi = 6.28318530717958647692f;
  const float log2e = 1.44269504088896340736f;

  for (int i = tid; i < M; i += NT) {
    float sn, cs;
    sincospif(-2.0f * (float)i / (float)Q, &sn, &cs);
    twQ[i] = make_float2(cs, sn);
  }
  for (int i = tid; i < M; i += NT) {
    // kWideFft: W_M^i (radix-4 passes); else W_M^{t k1} of the two-stage split
    const int e = kWideFft ? i : (i % P2) * (i / P2);
    float sn, cs;
    sincospif(-2.0f * (float)e / (float)M, &sn, &cs);
    tw1[i] = make_float2(cs, sn);
  }
  for (int i = tid; i < 2 * TB * (HP - H) * S; i += NT) {
    const int slot = i / ((HP - H) * S), rem = i % ((HP - H) * S);
    tbuf[(size_t)slot * HP * S + (size_t)H * S + rem] = make_float2(0.f, 0.f);
  }

  const int nstr = str1 - str0;
  const int nbatch = (nstr + TB - 1) / TB;
  const int tsz2 = H * S / 2;
  auto issue_batch = [&](int b, int buf) {
    const int j0 = str0 + b * TB;
    const int nb = min(TB, str1 - j0);
    for (int jj = 0; jj < nb; ++jj) {
      const float2* src = p.str + (size_t)(j0 + jj) * H * S;
      float2* dst = tbuf + (size_t)(buf * TB + jj) * HP * S;
      for (int i = tid; i < tsz2; i += NT) cp_async16(dst + 2 * i, src + 2 * i);
    }
    cp_async_commit();
  };

  const bool slot0 = (s == 0);
  const int ft = tid % F;

  for (int ps = 0; ps < nres; ps += RP) {
    float2 a[RT][HP], acc[RT][HP];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const int lr = ps + g * RT + i;
      const bool valid = lr < nres;
      const float2* src = p.res + ((size_t)(res0 + (valid ? lr : 0)) * H) * S + s;
#pragma unroll
      for (int h = 0; h < HP; ++h) {
        const float2 v = (valid && h < H) ? src[(size_t)h * S] : make_float2(0.f, 0.f);
        a[i][h] = make_float2(two_pi * v.x, two_pi * v.y);
        acc[i][h] = make_float2(0.f, 0.f);
      }
    }
    if (!kTmpl) {
      for (int rl = tid; rl < RP; rl += NT) {
        const int lr = ps + rl;
        const int n = (res0 + min(lr, nres - 1)) / T;
        rL[rl] = p.L[n];
        rG[rl] = p.gL[n];
      }
    }
    if (nbatch > 0) issue_batch(0, 0);
    for (int b = 0; b < nbatch; ++b) {
      const int cur = b & 1;
      if (b + 1 < nbatch) {
        issue_batch(b + 1, cur ^ 1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();  // streamed batch b landed
      const int j0 = str0 + b * TB;
      const int nb = min(TB, str1 - j0);
      if (kTmpl) {
        for (int jj = tid; jj < TB; jj += NT) {
          const int n = (j0 + min(jj, nb - 1)) / T;
          sL[jj] = p.L[n];
          sG[jj] = p.gL[n];
        }
      }

      // ---- Step 1 at slot s: Y = 2 pi sum_h conj(resident) streamed ----
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
            // resident = templates: X_hat = conj(Y) (the conjugate sits on the image)
            const float re = slot0 ? P[i] : P[i] + Qa[i];
            const float im = slot0 ? Qa[i] : (kTmpl ? Sa[i] - Ra[i] : Ra[i] - Sa[i]);
            spec[((g * RT + i) * TB + jj) * SP + s] = make_float2(re, im);
          }
        }
      }
      __syncthreads();  // spectra complete

      if constexpr (kWideFft) {
        // ---- per pair: X, P, and G(q) on 64 lanes ----
        constexpr int FW = 64, NSLOT = NT / FW, R4 = M / 4;
        const int slot = tid / FW, j = tid % FW;
#pragma unroll 1
        for (int pb = 0; pb < PAIRS; pb += NSLOT) {
          const int pr = pb + slot;
          if (pr < PAIRS) {  // slots without a pair skip (their barrier is not used)
            const int rl = pr / TB, jj = pr % TB;
            const bool ok = (jj < nb) && (ps + rl < nres);
            float2* sp = spec + (size_t)pr * SP;
            const int bar = 2 + slot;
            float2 v[4];
            // C2R pre-processing at k = j + 64 q, the inputs of the first pass
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int k = j + R4 * q;
              float2 A, B;
              if (k == 0) {
                const float2 s0 = sp[0];
                A = make_float2(s0.x, 0.f);
                B = make_float2(s0.y, 0.f);
              } else {
                A = sp[k];
                B = cconj(sp[M - k]);
              }
              const float2 d = cmul(csub(A, B), twQ[k]);
              v[q] = ok ? make_float2(A.x + B.x - d.y, A.y + B.y + d.x) : make_float2(0.f, 0.f);
            }
            named_sync(bar, FW);
            // forward transform: z(p) = X(2p) + i X(2p+1), p = j + 64 r after the last pass
            grad_radix4_pass<M, false, false, true>(sp, v, j, 1, tw1, bar);
            grad_radix4_pass<M, false, true, true>(sp, v, j, 4, tw1, bar);
            grad_radix4_pass<M, false, true, true>(sp, v, j, 16, tw1, bar);
            grad_radix4_pass<M, false, true, false>(sp, v, j, 64, tw1, bar);
            {
              const float Ln = kTmpl ? sL[jj] : rL[rl];
              const float gn = kTmpl ? sG[jj] : rG[rl];
              const float c = s2 * gn, cl = s2 * log2e, o = -Ln * log2e;
#pragma unroll
              for (int r = 0; r < 4; ++r)
                v[r] = make_float2(c * exp2f(fmaf(cl, v[r].x, o)), c * exp2f(fmaf(cl, v[r].y, o)));
            }
            // inverse transform: Y(k) = sum_mu p(mu) e^{+2 pi i mu k / M}, k = j + 64 r
            grad_radix4_pass<M, true, false, true>(sp, v, j, 1, tw1, bar);
            grad_radix4_pass<M, true, true, true>(sp, v, j, 4, tw1, bar);
            grad_radix4_pass<M, true, true, true>(sp, v, j, 16, tw1, bar);
            grad_radix4_pass<M, true, true, true>(sp, v, j, 64, tw1, bar);
            // G(k) = E(k) + e^{+2 pi i k / Q} O(k), E = (Y(k) + conj Y(M-k))/2, O = (Y(k) - conj Y(M-k))/(2i)
            float2 g[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              const int k = j + R4 * r;
              const float2 Yk = v[r];
              if (k == 0) {
                g[r] = make_float2(Yk.x + Yk.y, Yk.x - Yk.y);  // packed (G(0), G(Q/2))
              } else {
                const float2 Ym = cconj(sp[M - k]);
                const float2 E = make_float2(0.5f * (Yk.x + Ym.x), 0.5f * (Yk.y + Ym.y));
                const float2 O = make_float2(0.5f * (Yk.y - Ym.y), -0.5f * (Yk.x - Ym.x));
                g[r] = cadd(E, cmul(O, cconj(twQ[k])));
              }
            }
            named_sync(bar, FW);
#pragma unroll
            for (int r = 0; r < 4; ++r) sp[j + R4 * r] = g[r];
          }
        }
      } else {
        // ---- per pair: X, P, and G(q) on F lanes ----
#pragma unroll 1
        for (int pb = 0; pb < PAIRS; pb += PG) {
          const int pr = pb + tid / F;
          const int rl = pr / TB, jj = pr % TB;
          const bool ok = (pr < PAIRS) && (jj < nb) && (ps + rl < nres);
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
          if (ok) {
            const float Ln = kTmpl ? sL[jj] : rL[rl];
            const float gn = kTmpl ? sG[jj] : rG[rl];
            const float c = s2 * gn, cl = s2 * log2e, o = -Ln * log2e;
#pragma unroll
            for (int i = 0; i < RR; ++i) {
#pragma unroll
              for (int tp = 0; tp < P2; ++tp) y[i][tp] = sp[(ft * RR + i) * XP + tp];
              RegDft<P2>::run(y[i]);  // y[i][k2] = X(2p) + i X(2p+1), p = ft*RR + i + P1*k2
#pragma unroll
              for (int k2 = 0; k2 < P2; ++k2)
                y[i][k2] = make_float2(c * exp2f(fmaf(cl, y[i][k2].x, o)), c * exp2f(fmaf(cl, y[i][k2].y, o)));
              RegDft<P2, true>::run(y[i]);  // y[i][t] = sum_k2 e^{+2 pi i k2 t / P2} p(k1 + P1 k2)
            }
          }
          __syncwarp();
          if (ok) {
#pragma unroll
            for (int i = 0; i < RR; ++i)
#pragma unroll
              for (int t = 0; t < P2; ++t) sp[(ft * RR + i) * XP + t] = y[i][t];
          }
          __syncwarp();
          if (ok) {
#pragma unroll
            for (int k1 = 0; k1 < P1; ++k1) z[k1] = cmul(sp[k1 * XP + ft], cconj(tw1[k1 * P2 + ft]));
            RegDft<P1, true>::run(z);  // z[s'] = Y(ft + P2 s'), Y(k) = sum_mu p(mu) e^{+2 pi i mu k / M}
          }
          __syncwarp();
          if (ok) {
#pragma unroll
            for (int q1 = 0; q1 < P1; ++q1) sp[ft + P2 * q1] = z[q1];
          }
          __syncwarp();
          if (ok) {
            // G(k) = E(k) + e^{+2 pi i k / Q} O(k), E = (Y(k) + conj Y(M-k))/2, O = (Y(k) - conj Y(M-k))/(2i)
#pragma unroll
            for (int q1 = 0; q1 < P1; ++q1) {
              const int k = ft + P2 * q1;
              const float2 Yk = z[q1];
              if (q1 == 0 && ft == 0) {
                z[0] = make_float2(Yk.x + Yk.y, Yk.x - Yk.y);  // packed (G(0), G(Q/2))
              } else {
                const float2 Ym = cconj(sp[M - k]);
                const float2 E = make_float2(0.5f * (Yk.x + Ym.x), 0.5f * (Yk.y + Ym.y));
                const float2 O = make_float2(0.5f * (Yk.y - Ym.y), -0.5f * (Yk.x - Ym.x));
                z[q1] = cadd(E, cmul(O, cconj(twQ[k])));
              }
            }
          }
          __syncwarp();
          if (ok) {
#pragma unroll
            for (int q1 = 0; q1 < P1; ++q1) sp[ft + P2 * q1] = z[q1];
          }
        }
      }
      __syncthreads();  // G spectra complete

      // ---- gradient contraction at slot s ----
#pragma unroll 1
      for (int jj = 0; jj < TB; ++jj) {
        if (jj < nb) {
          const float2* bp = tb + (size_t)jj * HP * S;
          float A1[RT], A2[RT], A3[RT], A4[RT];
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            const float2 Gv = spec[((g * RT + i) * TB + jj) * SP + s];
            // re += S.x A1 + S.y A2 ; im += S.y A3 + S.x A4
            if (slot0) {
              A1[i] = Gv.x; A2[i] = 0.f; A3[i] = Gv.y; A4[i] = 0.f;
            } else if (kTmpl) {  // S * G
              A1[i] = Gv.x; A2[i] = -Gv.y; A3[i] = Gv.x; A4[i] = Gv.y;
            } else {             // S * conj(G)
              A1[i] = Gv.x; A2[i] = Gv.y; A3[i] = Gv.x; A4[i] = -Gv.y;
            }
          }
#pragma unroll
          for (int h = 0; h < HP; ++h) {
            const float2 bv = bp[h * S];
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              acc[i][h].x = fmaf(bv.x, A1[i], fmaf(bv.y, A2[i], acc[i][h].x));
              acc[i][h].y = fmaf(bv.y, A3[i], fmaf(bv.x, A4[i], acc[i][h].y));
            }
          }
        }
      }
      __syncthreads();  // streamed buffer `cur` and spectra free for reuse
    }
    // ---- write the gradient of the resident objects ----
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const int lr = ps + g * RT + i;
      if (lr < nres) {
        float2* dst = p.out + ((size_t)split * p.n_res + res0 + lr) * H * S + s;
#pragma unroll
        for (int h = 0; h < HP; ++h)
          if (h < H) dst[(size_t)h * S] = make_float2(two_pi * acc[i][h].x, two_pi * acc[i][h].y);
      }
    }
  }
}

template <int S, int HP>
int launch_grad_cfg(bool tmpl, const GradParams& p0, int IMGT, cudaStream_t stream) {
  using C = GradCfg<S, HP>;
  if constexpr (!C::kFits) {
    return RSVD_EUNSUPPORTED;
  } else {
    GradParams p = p0;
    if (!tmpl) {
      p.res_per_cta = images_per_cta(C::RP, p.T) * p.T;  // whole images, whole passes
      const long long grid = ((long long)p.n_res + p.res_per_cta - 1) / p.res_per_cta;
      if (cudaFuncSetAttribute(grad_kernel<S, HP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM) != cudaSuccess)
        return RSVD_ECUDA;
      grad_kernel<S, HP, false><<<(unsigned)grid, C::NT, C::SMEM, stream>>>(p);
    } else {
      p.res_per_cta = C::RP;
      const int groups = (p.n_res + C::RP - 1) / C::RP;
      dim3 grid(groups, p.nsplit);
      if (cudaFuncSetAttribute(grad_kernel<S, HP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)C::SMEM) != cudaSuccess)
        return RSVD_ECUDA;
      grad_kernel<S, HP, true><<<grid, C::NT, C::SMEM, stream>>>(p);
    }
    (void)IMGT;
    return launch_status();
  }
}

template <int S>
int launch_grad_s(int HP, bool tmpl, const GradParams& p, cudaStream_t stream) {
  switch (HP) {
    case 8: return launch_grad_cfg<S, 8>(tmpl, p, 0, stream);
    case 12: return launch_grad_cfg<S, 12>(tmpl, p, 0, stream);
    case 16: return launch_grad_cfg<S, 16>(tmpl, p, 0, stream);
    case 24: return launch_grad_cfg<S, 24>(tmpl, p, 0, stream);
    case 32: return launch_grad_cfg<S, 32>(tmpl, p, 0, stream);
    default: return RSVD_EUNSUPPORTED;
  }
}

// Rows of resident templates per CTA (needed to size the split partials).
template <int S>
int grad_tmpl_rows(int HP) {
  switch (HP) {
    case 8: return GradCfg<S, 8>::RP;
    case 12: return GradCfg<S, 12>::RP;
    case 16: return GradCfg<S, 16>::RP;
    case 24: return GradCfg<S, 24>::RP;
    case 32: return GradCfg<S, 32>::RP;
    default: return 0;
  }
}

RSVD_HIDDEN int launch_grad_s64(int HP, bool tmpl, const GradParams& p, cudaStream_t stream);
RSVD_HIDDEN int launch_grad_s128(int HP, bool tmpl, const GradParams& p, cudaStream_t stream);
RSVD_HIDDEN int launch_grad_s256(int HP, bool tmpl, const GradParams& p, cudaStream_t stream);

}  // namespace rsvd
