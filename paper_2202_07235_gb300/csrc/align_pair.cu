// Per-pair scoring kernel: one CTA per (image n, template j), looping over the
// T translations. Used by rsvd_align_scores (writes the full landscape X) and
// as the generic path of rsvd_align_best for sizes the fused kernel does not
// cover.
//
// Eq. (image_innerproduct_pm), Step 1: X_hat(q) = 2 pi sum_h conj(a_h(q)) b_h(q) for
// the half spectrum q = 0..Q/2 (slot s holds q = s; slot 0 packs q = 0 and q = Q/2).
// Step 2: X(gamma_m) = sum_{q<Q} e^{-2 pi i q m / Q} X_hat(q) with X_hat Hermitian, computed
// as a Q/2-point complex FFT of
//   Z(k) = [X_hat(k) + conj(X_hat(Q/2-k))] + i W_Q^k [X_hat(k) - conj(X_hat(Q/2-k))],
// whose output z(p) = X(gamma_{2p}) + i X(gamma_{2p+1}).
#include <math.h>

#include "align_common.cuh"

namespace rsvd {
namespace {

struct PairParams {
  const float2* cA;  // [N_A*T][H][Q/2]
  const float2* cB;  // [N_B][H][Q/2]
  float* X;          // [N_A][T][N_B][P Q] (scores mode; [K][T][P Q] with a pair list)
  float* best;       // [N_A][N_B] (reduce mode; [K] with a pair list)
  int32_t* arg;
  float* lse;        // nullable
  const int32_t* pairs;  // nullable: [K][2] (image, template) pairs, one CTA each
  int* status;
  int N_A, T, N_B, H, Q, P, log2M;  // output grid P Q angles, transform length M = P Q / 2
  float inv_sigma2;
};

constexpr int kMaxThreads = 512;

__device__ __forceinline__ int brev_bits(int i, int bits) {
  return bits == 0 ? 0 : (int)(__brev((unsigned)i) >> (32 - bits));
}

template <bool kReduce>
__global__ void __launch_bounds__(kMaxThreads) pair_kernel(const __grid_constant__ PairParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Mc = p.Q / 2;          // stored slots
  const int Qf = p.P * p.Q;        // output angles
  const int M = Qf / 2;            // transform length
  float2* spec = reinterpret_cast<float2*>(smem_raw);  // [M] half spectrum on the output grid
  float2* z = spec + M;                                  // [M]
  float2* twQ = z + M;                                   // [M]  W_Q^k
  float* red_v = reinterpret_cast<float*>(twQ + M);      // [32]
  int* red_i = reinterpret_cast<int*>(red_v + 32);       // [32]
  float* red_m = reinterpret_cast<float*>(red_i + 32);   // [32]
  float* red_l = red_m + 32;                             // [32]

  const long long pair = blockIdx.x;
  int n, j;
  if (p.pairs) {
    n = p.pairs[2 * pair];
    j = p.pairs[2 * pair + 1];
    if (n < 0 || n >= p.N_A || j < 0 || j >= p.N_B) {  // bad pair: recorded, outputs untouched
      if (threadIdx.x == 0) record(p.status, kDevBounds);
      return;
    }
  } else {
    n = (int)(pair / p.N_B);
    j = (int)(pair % p.N_B);
    if (n >= p.N_A) return;
  }
  const int tid = threadIdx.x, nth = blockDim.x;
  const int H = p.H;
  const float two_pi = 6.28318530717958647692f;
  const bool want_lse = kReduce && (p.lse != nullptr);
  const float s2 = p.inv_sigma2;

  for (int i = tid; i < M; i += nth) {
    float sn, cs;
    sincospif(-2.0f * (float)i / (float)Qf, &sn, &cs);
    twQ[i] = make_float2(cs, sn);
  }

  float run_best = -INFINITY, run_lse_m = -INFINITY, run_lse_s = 0.0f;
  int run_idx = 0;

  for (int t = 0; t < p.T; ++t) {
    const size_t row = (size_t)n * p.T + t;
    // Step 1 on the stored half spectrum; on a finer output grid (P > 1) the
    // spectrum is zero-padded: slot 0 keeps X_hat(0), the Nyquist term
    // X_hat(Q/2) moves to slot Q/2 with half its weight (its other half is the
    // mirror at -Q/2), slots above are zero (section 2.4, after eq. image_innerproduct)
    for (int s = tid; s < M; s += nth) {
      if (s >= Mc) {
        if (s > Mc) spec[s] = make_float2(0.f, 0.f);
        continue;
      }
      float P = 0.f, Qs = 0.f, Rs = 0.f, Ss = 0.f;
      const float2* a = p.cA + row * H * Mc + s;
      const float2* b = p.cB + (size_t)j * H * Mc + s;
      for (int h = 0; h < H; ++h) {
        const float2 av = a[(size_t)h * Mc], bv = b[(size_t)h * Mc];
        P = fmaf(av.x, bv.x, P);
        Qs = fmaf(av.y, bv.y, Qs);
        Rs = fmaf(av.x, bv.y, Rs);
        Ss = fmaf(av.y, bv.x, Ss);
      }
      if (s != 0) {
        spec[s] = make_float2(two_pi * (P + Qs), two_pi * (Rs - Ss));
      } else if (p.P == 1) {
        spec[0] = make_float2(two_pi * P, two_pi * Qs);
      } else {
        spec[0] = make_float2(two_pi * P, 0.f);
        spec[Mc] = make_float2(0.5f * two_pi * Qs, 0.f);
      }
    }
    __syncthreads();
    // pre-processing into the Q/2-point FFT input (bit-reversed order)
    for (int k = tid; k < M; k += nth) {
      float2 A, B;
      if (k == 0) {
        A = make_float2(spec[0].x, 0.f);
        B = make_float2(spec[0].y, 0.f);
      } else {
        A = spec[k];
        B = cconj(spec[M - k]);
      }
      const float2 d = cmul(csub(A, B), twQ[k]);
      z[brev_bits(k, p.log2M)] = make_float2(A.x + B.x - d.y, A.y + B.y + d.x);
    }
    __syncthreads();
    for (int half = 1; half < M; half *= 2) {
      const int stride = M / half;  // W_{2 half}^pos = W_Q^{pos * stride}
      for (int bf = tid; bf < M / 2; bf += nth) {
        const int pos = bf % half, grp = bf / half;
        const int i0 = grp * 2 * half + pos, i1 = i0 + half;
        const float2 w = twQ[pos * stride];
        const float2 a = z[i0];
        const float2 bw = cmul(z[i1], w);
        z[i0] = cadd(a, bw);
        z[i1] = csub(a, bw);
      }
      __syncthreads();
    }
    if (!kReduce) {
      float* out = p.X + (p.pairs ? ((size_t)pair * p.T + t) : (row * p.N_B + j)) * (size_t)Qf;
      for (int q = tid; q < M; q += nth) {
        out[2 * q] = z[q].x;
        out[2 * q + 1] = z[q].y;
      }
    } else {
      float bv = -INFINITY, lm = -INFINITY, ls = 0.f;
      int bi = 0x7fffffff;
      for (int q = tid; q < M; q += nth) {
        const float x0 = z[q].x, x1 = z[q].y;
        const int m0 = 2 * q;
        if (x0 > bv || (x0 == bv && m0 < bi)) { bv = x0; bi = m0; }
        if (x1 > bv || (x1 == bv && m0 + 1 < bi)) { bv = x1; bi = m0 + 1; }
        if (want_lse) {
          lse_push(lm, ls, s2 * x0);
          lse_push(lm, ls, s2 * x1);
        }
      }
      // warp reduce then block reduce
      argmax_warp_reduce(bv, bi, 32);
      if (want_lse) lse_warp_reduce(lm, ls, 32);
      const int warp = tid / 32, lane = tid % 32, nw = (nth + 31) / 32;
      if (lane == 0) {
        red_v[warp] = bv;
        red_i[warp] = bi;
        red_m[warp] = lm;
        red_l[warp] = ls;
      }
      __syncthreads();
      if (tid == 0) {
        float tb = red_v[0], tm = red_m[0], tl = red_l[0];
        int ti = red_i[0];
        for (int w = 1; w < nw; ++w) {
          if (red_v[w] > tb || (red_v[w] == tb && red_i[w] < ti)) { tb = red_v[w]; ti = red_i[w]; }
          if (want_lse) lse_merge(tm, tl, red_m[w], red_l[w]);
        }
        const int idx = t * Qf + ti;
        // translations are visited in increasing t, so an equal value keeps
        // the earlier (smaller) index t*Q + m
        if (t == 0 || tb > run_best) {
          run_best = tb;
          run_idx = idx;
        }
        if (want_lse) lse_merge(run_lse_m, run_lse_s, tm, tl);
      }
    }
    __syncthreads();
  }
  if (kReduce && tid == 0) {
    const size_t o = p.pairs ? (size_t)pair : (size_t)n * p.N_B + j;
    p.best[o] = run_best;
    p.arg[o] = run_idx;
    if (want_lse) p.lse[o] = run_lse_m + logf(run_lse_s);
  }
}

size_t pair_smem(int Qf) { return (size_t)3 * (Qf / 2) * sizeof(float2) + 4 * 32 * sizeof(float); }

int launch_pair(bool reduce, const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, float inv_sigma2,
                float* X, float* best, int32_t* arg, float* lse, cudaStream_t stream, int P = 1,
                const int32_t* pairs = nullptr, long long npairs = 0) {
  PairParams p{};
  p.pairs = pairs;
  p.P = P;
  p.cA = static_cast<const float2*>(cA);
  p.cB = static_cast<const float2*>(cB);
  p.X = X;
  p.best = best;
  p.arg = arg;
  p.lse = lse;
  p.status = status_word();
  p.N_A = N_A;
  p.T = T;
  p.N_B = N_B;
  p.H = H;
  p.Q = Q;
  int lg = 0;
  while ((1 << lg) < P * Q / 2) ++lg;
  p.log2M = lg;
  p.inv_sigma2 = inv_sigma2;
  const int M = P * Q / 2;
  int nth = ((M + 31) / 32) * 32;
  if (nth > kMaxThreads) nth = kMaxThreads;
  const long long blocks = pairs ? npairs : (long long)N_A * N_B;
  if (blocks > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
  if (blocks == 0) return RSVD_OK;
  const size_t smem = pair_smem(P * Q);
  if (reduce)
    pair_kernel<true><<<(unsigned)blocks, nth, smem, stream>>>(p);
  else
    pair_kernel<false><<<(unsigned)blocks, nth, smem, stream>>>(p);
  return launch_status();
}

}  // namespace

RSVD_HIDDEN int align_best_pairwise(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                    float inv_sigma2, float* best, int32_t* arg, float* lse, cudaStream_t stream) {
  return launch_pair(true, cA, N_A, T, cB, N_B, H, Q, inv_sigma2, nullptr, best, arg, lse, stream);
}

}  // namespace rsvd

namespace {

// P in {1, 2, 4, 8} with P Q <= 1024.
int check_fine(int Q, int P) {
  if (!(P == 1 || P == 2 || P == 4 || P == 8)) return RSVD_EUNSUPPORTED;
  if ((long long)P * Q > rsvd::kMaxQ) return RSVD_EUNSUPPORTED;
  return RSVD_OK;
}

}  // namespace

extern "C" int rsvd_align_scores_fine(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                                      int precision, float* X, void* stream) {
  using namespace rsvd;
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if ((rc = check_fine(Q, P)) != RSVD_OK) return rc;
  if (!X) return RSVD_EINVAL;
  return launch_pair(false, cA, N_A, T, cB, N_B, H, Q, 0.f, X, nullptr, nullptr, nullptr,
                     static_cast<cudaStream_t>(stream), P);
}

extern "C" int rsvd_align_best_fine(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                                    int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                                    void* stream) {
  using namespace rsvd;
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if ((rc = check_fine(Q, P)) != RSVD_OK) return rc;
  if (!best || !arg) return RSVD_EINVAL;
  if (lse && !(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
  return launch_pair(true, cA, N_A, T, cB, N_B, H, Q, inv_sigma2, nullptr, best, arg, lse,
                     static_cast<cudaStream_t>(stream), P);
}

extern "C" int rsvd_align_best_pairs(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                                     int precision, const int32_t* pairs, int K, float inv_sigma2, float* best,
                                     int32_t* arg, float* lse, void* stream) {
  using namespace rsvd;
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if ((rc = check_fine(Q, P)) != RSVD_OK) return rc;
  if (K < 0 || (K > 0 && (!pairs || !best || !arg))) return RSVD_EINVAL;
  if (lse && !(inv_sigma2 > 0.0f && isfinite(inv_sigma2))) return RSVD_EINVAL;
  if (((uintptr_t)pairs & 7u)) return RSVD_EINVAL;
  return launch_pair(true, cA, N_A, T, cB, N_B, H, Q, inv_sigma2, nullptr, best, arg, lse,
                     static_cast<cudaStream_t>(stream), P, pairs, K);
}

extern "C" int rsvd_align_scores(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                                 float* X, void* stream) {
  using namespace rsvd;
  if (precision != RSVD_FP32) {
    int rc = check_tc_args(cA, N_A, T, cB, N_B, H, Q, precision);
    if (rc != RSVD_OK) return rc;
    if (!X) return RSVD_EINVAL;
    return align_tc(cA, N_A, T, cB, N_B, H, Q, precision, 0.0f, nullptr, nullptr, nullptr, X,
                    static_cast<cudaStream_t>(stream));
  }
  int rc = check_align_args(cA, N_A, T, cB, N_B, H, Q, precision);
  if (rc != RSVD_OK) return rc;
  if (!X) return RSVD_EINVAL;
  return launch_pair(false, cA, N_A, T, cB, N_B, H, Q, 0.f, X, nullptr, nullptr, nullptr,
                     static_cast<cudaStream_t>(stream));
}
