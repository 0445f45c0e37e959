// Tensor-core scoring for the reduced-precision operand forms (operand.cuh):
// rsvd_align_best and rsvd_align_scores with RSVD_BF16, RSVD_FP16, RSVD_BF16X3,
// RSVD_FP16X3.
//
// Eq. (image_innerproduct_pm):
//   Step 1  X_hat(q) = 2 pi sum_h conj(a_h(q)) b_h(q)      -> tcgen05.mma into TMEM
//   Step 2  X(gamma_m) = sum_q e^{-i q gamma_m} X_hat(q)   -> per-thread FFT read from TMEM
// followed by the max / argmax / log-sum-exp over (gamma, delta) of
// sections 2.6-2.7, or the full X.
//
// Work item: a tile of 128 image rows (objects x translations, operand.cuh)
// against NT = 512 / Q templates. TMEM (128 lanes x 512 FP32 columns) holds the
// whole half spectrum of the 128 x NT pairs: lane = image row, column =
// 16 * group + (template, slot in group, re/im).
//
// Step 1 as real products of (re, im) components. For each of the 32 slot
// groups, one MMA chain D[128 x 16] += A[128 x K] * B[16 x K]^T with
//   A row    = the image row's components of the group's g slots (k = u 2Hp + 2h + c),
//   B row    = (template jj, slot u, c_out): zero outside the K range of slot u,
//              (b_re, b_im) for c_out = re and (b_im, -b_re) for c_out = im
//              (slot 0: (b(0), 0) and (0, b(Q/2)), the two real terms),
// so D(row, (jj, u, re)) = Re sum_h conj(a) b and D(.., im) = Im sum_h conj(a) b.
// The block-diagonal B is built in shared memory by the producer warp from the
// template rows; A arrives by bulk copy (TMA) of the row tile's operand block.
// Split-bf16x3 accumulates A_hi B_hi + A_hi B_lo + A_lo B_hi in the same
// FP32 accumulator.
//
// Step 2 (per thread = one (image row, template) pair, reading only its own
// TMEM lane): the real Q-point transform of the half spectrum as a complex
// M = Q/2 point DFT of
//   Z(k) = [X_hat(k) + conj X_hat(M - k)] + i W_Q^k [X_hat(k) - conj X_hat(M - k)],
//   z(p) = sum_k Z(k) W_M^{kp} = X(2p) + i X(2p + 1),
// split as M = g x 32 with k = k1 + 32 u, p = p1 + g p2: group k1 of TMEM holds
// exactly the g inputs k1 + 32 u of one first-stage DFT (and pairs with group
// 32 - k1 for the conjugate terms); first-stage results (twiddled by
// W_M^{k1 p1}) go back to the same columns, then each second-stage 32-point DFT
// gathers column 2 p1 of every group.
//
// Roles: warps 0 and 10 producers (alternate groups, one template-row copy
// each), warp 1 TMEM allocation + MMA issue (one elected lane of the converged
// warp), warps 2..9 epilogue (two warps per TMEM lane quadrant). Every wait is
// bounded (status word + abort flag; no role can hang the others).
#include <math.h>

#include "align_common.cuh"
#include "operand.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

constexpr int kTcThreads = 352;  // warps 0, 10 producers; 1 MMA; 2..9 epilogue
constexpr int kEpiThreads = 256;
constexpr long long kTcBudget = 1LL << 31;  // clock cycles per bounded wait
constexpr int kBarEpi = 1;
constexpr int kBarEpiStage = 2;  // between the two Step-2 stages of shared pairs (Q = 512)
constexpr int kTmemCols = 512;

template <int Q>
struct TcCfg {
  static constexpr int M = Q / 2;      // points of the half-length DFT (= packed slots)
  static constexpr int g = Q / 64;     // slots per group
  static constexpr int NT = 512 / Q;   // templates per tile
  // templates per epilogue thread; at Q = 512 (one template per tile) the two
  // warps of a lane quadrant share each pair instead (kShare)
  static constexpr bool kShare = NT == 1;
  static constexpr int TPT = kShare ? 1 : NT / 2;
  static constexpr int RES = kShare ? 2 : NT;  // result slots per row and tile
  // stages per group: at Q = 512 a group's operand (K = 16 Hp components, 64 KB
  // per plane at H = 16) arrives in two stages of half its K range (Hp even)
  static constexpr int NSPL = Q == 512 ? 2 : 1;
};

struct TcParams {
  const uint16_t* a;  // image operand planes (hi, then lo)
  const uint16_t* b;  // template operand planes
  // RSVD_FP16X3: factors 2^-e of the image rows (n T + t) and of the templates
  // (null for the other forms)
  const float* sA;
  const float* sB;
  long long a_plane, b_plane;
  float* best;
  int32_t* arg;
  float* lse;
  float* X;
  int* status;
  int N_A, T, N_B, IPT, nRT, nTP, CH, nUnits;
  int K, KC, KS, Hp, stages, split, lse_on, nprod;
  int bres;  // template blocks of all 32 groups resident for a whole work unit (single-pass forms)
  float inv_sigma2;
  uint32_t idesc;
  // a_bytes, b_bytes: one stage's A and B blocks per plane (a group's part of K)
  uint32_t stage_bytes, a_bytes, b_bytes, dense_off, dense_bytes, bres_off, res_off, bar_off;
  float2 WQ[256];  // W_Q^k = exp(-2 pi i k / Q), k < Q/2
  float2 WM[256];  // W_M^k, M = Q/2
};

// Bounded wait for a barrier phase. The abort flag and the clock are checked
// every 16 polls; `sleep_ns` > 0 backs off between polls (long waits of many
// threads, which would otherwise keep the shared-memory pipe busy).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag, int* status,
                                        unsigned sleep_ns = 0) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (unsigned n = 1;; ++n) {
    if (sleep_ns) __nanosleep(sleep_ns);
    if (mbar_try_wait(bar, parity)) return true;
    if ((n & 15u) == 0u) {
      if (*abort_flag) return false;
      if (clock64() - t0 > kTcBudget) {
        record(status, kDevTimeout);
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// The MMA chain of one group: K-steps ks = 0..KS-1 (descriptor start addresses
// advance by a_step / b_step), bf16x3 adding the A_hi B_lo and A_lo B_hi terms.
// `acc0` = 1 when the chain continues a group's accumulation from an earlier stage.
template <int KS, bool kSplit>
__device__ __forceinline__ void issue_group(uint32_t leader, uint32_t d, uint64_t ad, uint64_t bd, uint64_t ad_lo,
                                            uint64_t bd_lo, uint64_t a_step, uint64_t b_step, uint32_t idesc,
                                            uint32_t acc0) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    tc_mma_f16_by(leader, d, ad + ks * a_step, bd + ks * b_step, idesc, (ks > 0 || acc0) ? 1u : 0u);
    if (kSplit) {
      tc_mma_f16_by(leader, d, ad + ks * a_step, bd_lo + ks * b_step, idesc, 1u);
      tc_mma_f16_by(leader, d, ad_lo + ks * a_step, bd + ks * b_step, idesc, 1u);
    }
  }
}

// Single-pass chains of two groups with their K-steps interleaved (each chain
// accumulates into its own TMEM columns, so consecutive MMAs never wait on one
// another's accumulator).
template <int KS>
__device__ __forceinline__ void issue_two_groups(uint32_t leader, uint32_t d0, uint32_t d1, uint64_t ad0, uint64_t bd0,
                                                 uint64_t ad1, uint64_t bd1, uint64_t a_step, uint64_t b_step,
                                                 uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < KS; ++ks) {
    tc_mma_f16_by(leader, d0, ad0 + ks * a_step, bd0 + ks * b_step, idesc, ks > 0 ? 1u : 0u);
    tc_mma_f16_by(leader, d1, ad1 + ks * a_step, bd1 + ks * b_step, idesc, ks > 0 ? 1u : 0u);
  }
}

__device__ __forceinline__ void issue_two_groups_rt(int KS, uint32_t leader, uint32_t d0, uint32_t d1, uint64_t ad0,
                                                    uint64_t bd0, uint64_t ad1, uint64_t bd1, uint64_t a_step,
                                                    uint64_t b_step, uint32_t idesc) {
  switch (KS) {
    case 2: issue_two_groups<2>(leader, d0, d1, ad0, bd0, ad1, bd1, a_step, b_step, idesc); return;
    case 3: issue_two_groups<3>(leader, d0, d1, ad0, bd0, ad1, bd1, a_step, b_step, idesc); return;
    case 4: issue_two_groups<4>(leader, d0, d1, ad0, bd0, ad1, bd1, a_step, b_step, idesc); return;
    case 6: issue_two_groups<6>(leader, d0, d1, ad0, bd0, ad1, bd1, a_step, b_step, idesc); return;
    case 8: issue_two_groups<8>(leader, d0, d1, ad0, bd0, ad1, bd1, a_step, b_step, idesc); return;
    default:
      for (int ks = 0; ks < KS; ++ks) {
        tc_mma_f16_by(leader, d0, ad0 + ks * a_step, bd0 + ks * b_step, idesc, ks > 0 ? 1u : 0u);
        tc_mma_f16_by(leader, d1, ad1 + ks * a_step, bd1 + ks * b_step, idesc, ks > 0 ? 1u : 0u);
      }
  }
}

template <bool kSplit>
__device__ __forceinline__ void issue_group_rt(int KS, uint32_t leader, uint32_t d, uint64_t ad, uint64_t bd,
                                               uint64_t ad_lo, uint64_t bd_lo, uint64_t a_step, uint64_t b_step,
                                               uint32_t idesc, uint32_t acc0) {
  switch (KS) {
    case 2: issue_group<2, kSplit>(leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, idesc, acc0); return;
    case 3: issue_group<3, kSplit>(leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, idesc, acc0); return;
    case 4: issue_group<4, kSplit>(leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, idesc, acc0); return;
    case 6: issue_group<6, kSplit>(leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, idesc, acc0); return;
    case 8: issue_group<8, kSplit>(leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, idesc, acc0); return;
    default:
      for (int ks = 0; ks < KS; ++ks) {
        tc_mma_f16_by(leader, d, ad + ks * a_step, bd + ks * b_step, idesc, (ks > 0 || acc0) ? 1u : 0u);
        if (kSplit) {
          tc_mma_f16_by(leader, d, ad + ks * a_step, bd_lo + ks * b_step, idesc, 1u);
          tc_mma_f16_by(leader, d, ad_lo + ks * a_step, bd + ks * b_step, idesc, 1u);
        }
      }
  }
}

// Z(k) = [X + conj P] + i w [X - conj P]
__device__ __forceinline__ float2 zform(float2 X, float2 P, float2 w) {
  const float2 A = make_float2(X.x + P.x, X.y - P.y);
  const float2 B = make_float2(X.x - P.x, X.y + P.y);
  const float2 C = cmul(w, B);
  return make_float2(A.x - C.y, A.y + C.x);
}

// Step 2, first stage, for group pairs k1 = K1B .. K1E-1 of one (image row,
// template jj) pair: pre-processing, g-point DFTs, twiddles; in place. The
// loads of the next group pair are in flight while this one is computed.
template <int Q, int K1B, int K1E>
__device__ __forceinline__ void tc_first_stage(const TcParams& p, uint32_t tl, uint32_t cb) {
  constexpr int g = TcCfg<Q>::g;
  uint32_t cur[4 * g], nxt[4 * g];
  tmem_ld_pair_issue<g>(tl + K1B * 16 + cb, tl + ((32 - K1B) & 31) * 16 + cb, cur);
  tmem_wait_ld_tie<4 * g>(cur);
#pragma unroll
  for (int k1 = K1B; k1 < K1E; ++k1) {
    const int k2 = (32 - k1) & 31;
    if (k1 + 1 < K1E) tmem_ld_pair_issue<g>(tl + (k1 + 1) * 16 + cb, tl + ((31 - k1) & 31) * 16 + cb, nxt);
    float2 xa[g], xb[g], za[g], zb[g];
#pragma unroll
    for (int i = 0; i < g; ++i) {
      xa[i] = make_float2(__uint_as_float(cur[2 * i]), __uint_as_float(cur[2 * i + 1]));
      xb[i] = make_float2(__uint_as_float(cur[2 * g + 2 * i]), __uint_as_float(cur[2 * g + 2 * i + 1]));
    }
    if (k1 == 0) {
      za[0] = make_float2(xa[0].x + xa[0].y, xa[0].x - xa[0].y);  // X_hat(0), X_hat(M) real
#pragma unroll
      for (int u = 1; u < g; ++u) za[u] = zform(xa[u], xa[g - u], p.WQ[32 * u]);
    } else if (k1 == 16) {
#pragma unroll
      for (int u = 0; u < g; ++u) za[u] = zform(xa[u], xa[g - 1 - u], p.WQ[16 + 32 * u]);
    } else {
#pragma unroll
      for (int u = 0; u < g; ++u) {
        const float2 X = xa[u], P = xb[g - 1 - u];
        const float2 A = make_float2(X.x + P.x, X.y - P.y);
        const float2 B = make_float2(X.x - P.x, X.y + P.y);
        const float2 Cw = cmul(p.WQ[k1 + 32 * u], B);
        za[u] = make_float2(A.x - Cw.y, A.y + Cw.x);          // A + i C
        zb[g - 1 - u] = make_float2(A.x + Cw.y, Cw.x - A.y);  // conj(A) + i conj(C): k' = M - k
      }
    }
    RegDft<g>::run(za);
#pragma unroll
    for (int p1 = 1; p1 < g; ++p1) za[p1] = cmul(za[p1], p.WM[k1 * p1]);
    tmem_st<g>(tl + k1 * 16 + cb, za);
    if (k2 != k1) {
      RegDft<g>::run(zb);
#pragma unroll
      for (int p1 = 1; p1 < g; ++p1) zb[p1] = cmul(zb[p1], p.WM[k2 * p1]);
      tmem_st<g>(tl + k2 * 16 + cb, zb);
    }
    if (k1 + 1 < K1E) {
      tmem_wait_ld_tie<4 * g>(nxt);
#pragma unroll
      for (int i = 0; i < 4 * g; ++i) cur[i] = nxt[i];
    }
  }
}

// Step 2, second stage, for p1 = P1B .. P1E-1: 32-point DFTs over k1 (column
// 2 p1 of every group) and the reductions. Returns (max of X / 2pi over those
// m, its m, lse max, lse sum) with the lse in units of inv_sigma2 * X; writes
// X instead when kWriteX.
template <int Q, bool kWriteX, int P1B, int P1E>
__device__ __forceinline__ float4 tc_second_stage(const TcParams& p, uint32_t tl, uint32_t cb, bool row_ok,
                                                  float* xrow, float sc) {
  constexpr int g = TcCfg<Q>::g;
  constexpr float kTwoPi = 6.283185307179586f;
  // sc: the pair's power-of-two factor (RSVD_FP16X3), exact on every value
  const float cs = kTwoPi * p.inv_sigma2 * sc, xs = kTwoPi * sc;
  float best = -INFINITY, lm = -INFINITY, ls = 0.0f;
  int bm = 0;
#pragma unroll
  for (int p1 = P1B; p1 < P1E; ++p1) {
    float2 z[32];
    {
      uint32_t r[4][16];  // all 32 loads of the pass in flight, then one wait
#pragma unroll
      for (int b8 = 0; b8 < 4; ++b8) tmem_ld2x8_issue(tl + (uint32_t)(b8 * 8 * 16) + cb + 2 * p1, 16, r[b8]);
#pragma unroll
      for (int b8 = 0; b8 < 4; ++b8) tmem_wait_ld_tie<16>(r[b8]);
#pragma unroll
      for (int b8 = 0; b8 < 4; ++b8)
#pragma unroll
        for (int i = 0; i < 8; ++i) z[b8 * 8 + i] = make_float2(__uint_as_float(r[b8][2 * i]), __uint_as_float(r[b8][2 * i + 1]));
    }
    RegDft<32>::run(z);  // z[p2] = X(2p) + i X(2p+1) over 2 pi, p = p1 + g p2
    if (kWriteX) {
      if (row_ok) {
#pragma unroll
        for (int p2 = 0; p2 < 32; ++p2)
          *reinterpret_cast<float2*>(xrow + 2 * (p1 + g * p2)) = make_float2(xs * z[p2].x, xs * z[p2].y);
      }
    } else {
      float v[64];
#pragma unroll
      for (int p2 = 0; p2 < 32; ++p2) {
        v[2 * p2] = z[p2].x;
        v[2 * p2 + 1] = z[p2].y;
      }
      float pb;
      int pi;
      tree_argmax<64>(v, pb, pi);  // m increases with the index within a pass
      const int m = 2 * p1 + 2 * g * (pi >> 1) + (pi & 1);
      if (pb > best || (pb == best && m < bm)) {
        best = pb;
        bm = m;
      }
      if (p.lse_on) {
        const float off = pb * cs;
        float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < 64; ++i) acc[i & 3] += __expf(fmaf(v[i], cs, -off));
        lse_merge(lm, ls, off, (acc[0] + acc[1]) + (acc[2] + acc[3]));
      }
    }
  }
  return make_float4(best * sc, __int_as_float(bm), lm, ls);
}

// Step 2 and the per-row reduction for one (image row, template jj) pair by
// one thread (Q <= 256): the real Q-point transform of the half spectrum as a
// complex M = Q/2 point DFT of
//   Z(k) = [X_hat(k) + conj X_hat(M - k)] + i W_Q^k [X_hat(k) - conj X_hat(M - k)],
// split as M = g x 32 (see the file header).
template <int Q, bool kWriteX>
__device__ __forceinline__ float4 tc_pair(const TcParams& p, uint32_t tl, int jj, bool row_ok, float* xrow,
                                          float sc) {
  constexpr int g = TcCfg<Q>::g;
  const uint32_t cb = (uint32_t)(jj * 2 * g);
  tc_first_stage<Q, 0, 17>(p, tl, cb);
  tmem_wait_st();
  return tc_second_stage<Q, kWriteX, 0, g>(p, tl, cb, row_ok, xrow, sc);
}

// The same at Q = 512 (one template per tile) shared by the two warps of a
// lane quadrant: warp `sub` takes group pairs k1 = 0..8 (sub 0) or 9..16
// (sub 1) of the first stage and p1 = 0..3 or 4..7 of the second; between the
// stages every epilogue thread meets at a named barrier. Returns the partial
// reduction over this warp's angles.
template <int Q, bool kWriteX>
__device__ __forceinline__ float4 tc_pair_shared(const TcParams& p, uint32_t tl, int sub, bool row_ok, float* xrow,
                                                 float sc) {
  constexpr int g = TcCfg<Q>::g;
  static_assert(g == 8, "shared pairs are laid out for g = 8");
  if (sub == 0) tc_first_stage<Q, 0, 9>(p, tl, 0);
  else tc_first_stage<Q, 9, 17>(p, tl, 0);
  tmem_wait_st();
  tc_fence_before();
  named_sync(kBarEpiStage, kEpiThreads);
  tc_fence_after();
  if (sub == 0) return tc_second_stage<Q, kWriteX, 0, g / 2>(p, tl, 0, row_ok, xrow, sc);
  return tc_second_stage<Q, kWriteX, g / 2, g>(p, tl, 0, row_ok, xrow, sc);
}

// kPair: single-pass forms with resident template blocks (the producers only
// issue copies) take two groups from two consecutive stages per MMA step, their
// chains interleaved; the other plans keep one group per step.
template <int Q, bool kWriteX, bool kPair>
__global__ void __launch_bounds__(kTcThreads, 1) tc_align_kernel(const __grid_constant__ TcParams p) {
  using C = TcCfg<Q>;
  constexpr int g = C::g, NT = C::NT, TPT = C::TPT, NSPL = C::NSPL;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(tc_smem + p.bar_off);
  uint64_t* empty = full + p.stages;
  uint64_t* tmem_full = empty + p.stages;
  uint64_t* tmem_empty = tmem_full + 1;
  uint64_t* drain = tmem_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile uint32_t* abort_flag = tmem_slot + 1;
  // template rows [plane][jj][group][K], one copy per producer warp
  uint16_t* dense = reinterpret_cast<uint16_t*>(tc_smem + p.dense_off + (threadIdx.x >= 320 ? p.dense_bytes : 0u));
  float4* res = reinterpret_cast<float4*>(tc_smem + p.res_off);          // [2][RES][128]

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int planes = p.split ? 2 : 1;

  if (tid == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&full[s], 2);  // expect_tx arrival + arrival after the template block is written
      mbar_init(&empty[s], 1);
    }
    mbar_init(tmem_full, 1);
    mbar_init(tmem_empty, kEpiThreads);
    mbar_init(drain, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  // the template blocks' zeros never change: clear them once
  if (p.bres) {
    uint32_t* bz = reinterpret_cast<uint32_t*>(tc_smem + p.bres_off);
    for (int i = tid; i < (int)(kOpGroups * p.b_bytes / 4); i += kTcThreads) bz[i] = 0u;
  } else {
    for (int s = 0; s < p.stages; ++s) {
      uint32_t* bz = reinterpret_cast<uint32_t*>(tc_smem + (size_t)s * p.stage_bytes + planes * p.a_bytes);
      for (int i = tid; i < (int)(planes * p.b_bytes / 4); i += kTcThreads) bz[i] = 0u;
    }
  }
  fence_proxy_async_smem();
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 || (warp == 10 && p.nprod == 2)) {
    // ================= producers =================
    const long long mine = warp == 10 ? 1 : 0;  // with two producers, this warp fills the groups with it % 2 == mine
    // This lane's entries of the block-diagonal template operand, the same for
    // every group: source word in the template rows (group 0, plane 0),
    // destination word in the block, slot-0 flag (u == 0).
    constexpr int kMaxItems = 8;  // NT * g * Hp / 32 with Hp <= 32
    // With NSPL = 2 an item lies in one half of the group's K range (it_kh),
    // and its destination is relative to that half's block.
    int it_src[kMaxItems], it_dst[kMaxItems];
    uint32_t it_u0 = 0u, it_kh = 0u;
    const int n_items = NT * g * p.Hp;
    const int k_part = p.K / NSPL;
#pragma unroll
    for (int r = 0; r < kMaxItems; ++r) {
      const int i = lane + 32 * r;
      it_src[r] = -1;
      it_dst[r] = 0;
      if (i < n_items) {
        const int h = i % p.Hp;
        const int q = i / p.Hp;
        const int u = q % g, jj = q / g;
        const int k = u * 2 * p.Hp + 2 * h;
        const int kh = k / k_part, kl = k - kh * k_part;
        const int nr = jj * 2 * g + 2 * u;
        it_src[r] = (jj * kOpGroups * p.K + k) >> 1;
        it_dst[r] = ((((kl >> 3) * 16 + nr) * 8) + (kl & 7)) >> 1;
        if (u == 0) it_u0 |= 1u << r;
        if (kh) it_kh |= 1u << r;
      }
    }
    const uint32_t* dense_w = reinterpret_cast<const uint32_t*>(dense);
    const int dense_plane_w = NT * kOpGroups * p.K / 2;
    const int b_plane_w = (int)(p.b_bytes / 4);
    long long it = 0, ptile = 0;
    int ps = 0;            // stage of iteration it
    uint32_t pphase = 0u;  // parity of (it / stages)
    bool ok = true;
    for (int unit = blockIdx.x; unit < p.nUnits && ok; unit += gridDim.x) {
      const int tp = unit % p.nTP, chunk = unit / p.nTP;
      const int rt0 = chunk * p.CH, rt1 = min(p.nRT, rt0 + p.CH);
      // template rows of this template group (zeros past N_B)
      const int pieces = planes * NT * kOpGroups * p.KC;  // 16-byte pieces
      for (int base = 0; base < pieces; base += 8 * 32) {
        uint4 v[8];
        int dst[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {  // eight loads in flight per lane
          const int i = base + u * 32 + lane;
          v[u] = make_uint4(0u, 0u, 0u, 0u);
          dst[u] = -1;
          if (i < pieces) {
            const int kc = i % p.KC;
            int r = i / p.KC;
            const int grp = r % kOpGroups;
            r /= kOpGroups;
            const int jj = r % NT, pl = r / NT;
            const int j = tp * NT + jj;
            dst[u] = ((pl * NT + jj) * kOpGroups + grp) * p.K + kc * 8;
            if (j < p.N_B) {
              const uint16_t* src = p.b + pl * p.b_plane +
                                    ((((long long)(j >> 7) * kOpGroups + grp) * p.KC + kc) * kOpLanes + (j & 127)) * 8;
              v[u] = __ldg(reinterpret_cast<const uint4*>(src));
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (dst[u] >= 0) *reinterpret_cast<uint4*>(dense + dst[u]) = v[u];
      }
      __syncwarp();
      if (p.bres) {
        // resident template blocks of this warp's groups: rewritten only after every
        // MMA of the previous unit (the last tile committed to tmem_full) is done
        if (ptile > 0) {
          int w = 1;
          if (lane == 0) w = tc_wait(tmem_full, (uint32_t)((ptile - 1) & 1), abort_flag, p.status);
          if (!__shfl_sync(0xffffffffu, w, 0)) {
            ok = false;
            break;
          }
        }
        for (int grp = (int)mine; grp < kOpGroups; grp += p.nprod) {
          uint32_t* bp0 = reinterpret_cast<uint32_t*>(tc_smem + p.bres_off + (size_t)grp * p.b_bytes);
          const int gofs = grp * p.K / 2;
#pragma unroll
          for (int r = 0; r < kMaxItems; ++r) {
            if (it_src[r] < 0) continue;
            const uint32_t v = dense_w[gofs + it_src[r]];
            const bool slot0 = grp == 0 && ((it_u0 >> r) & 1u);
            bp0[it_dst[r]] = slot0 ? (v & 0x0000FFFFu) : v;
            bp0[it_dst[r] + 4] = slot0 ? (v & 0xFFFF0000u) : (__byte_perm(v, 0u, 0x1032) ^ 0x80000000u);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
      }
      for (int rt = rt0; rt < rt1 && ok; ++rt, ++ptile) {
        for (int gi = 0; gi < kOpGroups * NSPL; ++gi) {
          const int grp = gi / NSPL, kh = gi - grp * NSPL;  // group, part of its K range
          const int s = ps;
          if (p.nprod == 2 && (it & 1) != mine) {
            ++it;
            if (++ps == p.stages) {
              ps = 0;
              pphase ^= 1u;
            }
            continue;
          }
          if (it >= p.stages) {
            int w = 1;
            if (lane == 0) w = tc_wait(&empty[s], pphase ^ 1u, abort_flag, p.status);
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) {
              ok = false;
              break;
            }
          }
          unsigned char* st = tc_smem + (size_t)s * p.stage_bytes;
          if (lane == 0) {
            mbar_arrive_expect_tx(&full[s], planes * p.a_bytes);
            const long long off = (((long long)rt * kOpGroups + grp) * p.KC + (long long)kh * (p.KC / NSPL)) *
                                  kOpLanes * 8;
            for (int pl = 0; pl < planes; ++pl) bulk_g2s(st + pl * p.a_bytes, p.a + pl * p.a_plane + off, p.a_bytes, &full[s]);
          }
          // block-diagonal template operand: rows (jj, u, re/im), K-major core matrices
          uint32_t* bst = reinterpret_cast<uint32_t*>(st + planes * p.a_bytes);
          const int gofs = grp * p.K / 2;
#pragma unroll
          for (int r = 0; r < (p.bres ? 0 : kMaxItems); ++r) {
            if (it_src[r] < 0 || (int)((it_kh >> r) & 1u) != kh) continue;
            const bool slot0 = grp == 0 && ((it_u0 >> r) & 1u);
            for (int pl = 0; pl < planes; ++pl) {
              const uint32_t v = dense_w[pl * dense_plane_w + gofs + it_src[r]];
              uint32_t re_row, im_row;
              if (slot0) {  // slot 0: the real q = 0 and q = Q/2 terms
                re_row = v & 0x0000FFFFu;
                im_row = v & 0xFFFF0000u;
              } else {
                re_row = v;                                          // (b_re, b_im)
                im_row = __byte_perm(v, 0u, 0x1032) ^ 0x80000000u;  // (b_im, -b_re)
              }
              uint32_t* bp = bst + pl * b_plane_w + it_dst[r];
              bp[0] = re_row;
              bp[4] = im_row;  // next row: +8 elements
            }
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[s]);
          ++it;
          if (++ps == p.stages) {
            ps = 0;
            pphase ^= 1u;
          }
        }
      }
    }
    if (!ok && lane == 0) {
      // copies this warp issued that may still be in flight land before the CTA exits
      const long long first = it > p.stages ? it - p.stages : 0;
      for (long long k = first; k < it; ++k)
        if (p.nprod == 1 || (k & 1) == mine) mbar_wait_bounded(&full[k % p.stages], (uint32_t)((k / p.stages) & 1), kTcBudget);
    }
  } else if (warp == 10) {
    // second producer not used (its template-row copy does not fit)
  } else if (warp == 1) {
    // ================= MMA issue (converged warp, one elected lane issues) =================
    {
      const uint32_t mma_leader = elect_one();  // the same lane issues every MMA and commit
      long long it = 0, tile = 0;
      int ms = 0;
      uint32_t mphase = 0u;
      bool ok = true;
      constexpr uint32_t kSbo = 128;                 // 8 rows x 16 bytes
      const uint32_t a_lbo = kOpLanes * 16;          // next 8 components: 128 rows further
      const uint32_t b_lbo = 16 * 16;                // 16 template rows
      for (int unit = blockIdx.x; unit < p.nUnits && ok; unit += gridDim.x) {
        const int chunk = unit / p.nTP;
        const int rt0 = chunk * p.CH, rt1 = min(p.nRT, rt0 + p.CH);
        for (int rt = rt0; rt < rt1 && ok; ++rt) {
          if (tile > 0 && !__all_sync(0xffffffffu, tc_wait(tmem_empty, (uint32_t)((tile - 1) & 1), abort_flag, p.status))) {
            ok = false;
            break;
          }
          tc_fence_after();
          for (int grp = 0; kPair && grp < kOpGroups; grp += 2) {
            const int s0 = ms;
            const uint32_t ph0 = mphase;
            const int s1 = (ms + 1 == p.stages) ? 0 : ms + 1;
            const uint32_t ph1 = (ms + 1 == p.stages) ? (mphase ^ 1u) : mphase;
            if (!__all_sync(0xffffffffu, tc_wait(&full[s0], ph0, abort_flag, p.status)) ||
                !__all_sync(0xffffffffu, tc_wait(&full[s1], ph1, abort_flag, p.status))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t a_step = (2u * a_lbo) >> 4, b_step = (2u * b_lbo) >> 4;
            const uint64_t ad0 = smem_desc_kmajor(smem_addr(tc_smem + (size_t)s0 * p.stage_bytes), a_lbo, kSbo);
            const uint64_t ad1 = smem_desc_kmajor(smem_addr(tc_smem + (size_t)s1 * p.stage_bytes), a_lbo, kSbo);
            const uint64_t bd0 = smem_desc_kmajor(smem_addr(tc_smem + p.bres_off + (size_t)grp * p.b_bytes), b_lbo, kSbo);
            const uint64_t bd1 =
                smem_desc_kmajor(smem_addr(tc_smem + p.bres_off + (size_t)(grp + 1) * p.b_bytes), b_lbo, kSbo);
            issue_two_groups_rt(p.KS, mma_leader, tmem_base + (uint32_t)(grp * 16), tmem_base + (uint32_t)(grp * 16 + 16),
                                ad0, bd0, ad1, bd1, a_step, b_step, p.idesc);
            tc_commit_by(mma_leader, &empty[s0]);
            tc_commit_by(mma_leader, &empty[s1]);
            __syncwarp();
            it += 2;
            ms = (s1 + 1 == p.stages) ? 0 : s1 + 1;
            mphase = (s1 + 1 == p.stages) ? (ph1 ^ 1u) : ph1;
          }
          for (int gi = 0; !kPair && gi < kOpGroups * NSPL; ++gi) {
            const int grp = gi / NSPL, kh = gi - grp * NSPL;
            const int s = ms;
            if (!__all_sync(0xffffffffu, tc_wait(&full[s], mphase, abort_flag, p.status))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_addr(tc_smem + (size_t)s * p.stage_bytes);
            const uint32_t a_hi = st, a_lo = st + p.a_bytes;
            const uint32_t b_hi = p.bres ? smem_addr(tc_smem + p.bres_off + (size_t)grp * p.b_bytes)
                                         : st + planes * p.a_bytes;
            const uint32_t b_lo = b_hi + p.b_bytes;
            const uint32_t d = tmem_base + (uint32_t)(grp * 16);
            // descriptors of K-step 0; a K-step of 16 components advances the start
            // address by 2 core-matrix columns (the low field counts 16-byte units)
            const uint64_t ad = smem_desc_kmajor(a_hi, a_lbo, kSbo), bd = smem_desc_kmajor(b_hi, b_lbo, kSbo);
            const uint64_t a_step = (2u * a_lbo) >> 4, b_step = (2u * b_lbo) >> 4;
            const uint32_t leader = mma_leader;
            const uint32_t acc0 = kh > 0 ? 1u : 0u;  // later parts continue the group's accumulation
            if (!p.split) {
              issue_group_rt<false>(p.KS, leader, d, ad, bd, 0, 0, a_step, b_step, p.idesc, acc0);
            } else {
              const uint64_t ad_lo = smem_desc_kmajor(a_lo, a_lbo, kSbo), bd_lo = smem_desc_kmajor(b_lo, b_lbo, kSbo);
              issue_group_rt<true>(p.KS, leader, d, ad, bd, ad_lo, bd_lo, a_step, b_step, p.idesc, acc0);
            }
            tc_commit_by(leader, &empty[s]);
            __syncwarp();
            ++it;
            if (++ms == p.stages) {
              ms = 0;
              mphase ^= 1u;
            }
          }
          if (!ok) break;
          tc_commit_by(mma_leader, tmem_full);
          ++tile;
        }
      }
      tc_commit_by(mma_leader, drain);  // every MMA complete before TMEM is released
      mbar_wait_bounded(drain, 0, kTcBudget);
      __syncwarp();
    }
  } else {
    // ================= epilogue =================
    const int qd = warp & 3, sub = (warp - 2) >> 2;
    const int row = qd * 32 + lane;
    const int ep = tid - 64;
    const uint32_t tl = tmem_base + ((uint32_t)(qd * 32) << 16);
    const int n_local = row / p.T, t = row - n_local * p.T;
    long long tile = 0;
    bool run = true;
    for (int unit = blockIdx.x; unit < p.nUnits && run; unit += gridDim.x) {
      const int tp = unit % p.nTP, chunk = unit / p.nTP;
      const int rt0 = chunk * p.CH, rt1 = min(p.nRT, rt0 + p.CH);
      for (int rt = rt0; rt < rt1; ++rt, ++tile) {
        const bool got = tc_wait(tmem_full, (uint32_t)(tile & 1), abort_flag, p.status, 128);
        __syncwarp();
        tc_fence_after();
        const long long n = (long long)rt * p.IPT + n_local;
        const bool row_ok = got && row < p.IPT * p.T && n < p.N_A;
        float4 r[TPT];
#pragma unroll
        for (int i = 0; i < TPT; ++i) {
          const int jj = C::kShare ? 0 : sub * TPT + i;
          const int j = tp * NT + jj;
          float* xrow = nullptr;
          if (kWriteX) xrow = p.X + ((n * p.T + t) * (long long)p.N_B + j) * (Q);
          const bool ok = row_ok && j < p.N_B;
          const float sc = (p.sA != nullptr && ok) ? p.sA[n * p.T + t] * p.sB[j] : 1.0f;
          if constexpr (C::kShare) {
            r[i] = tc_pair_shared<Q, kWriteX>(p, tl, sub, ok, xrow, sc);
          } else {
            r[i] = tc_pair<Q, kWriteX>(p, tl, jj, ok, xrow, sc);
          }
        }
        tc_fence_before();
        mbar_arrive(tmem_empty);
        if (!kWriteX) {
          float4* rb = res + (size_t)(tile & 1) * C::RES * kOpLanes;
#pragma unroll
          for (int i = 0; i < TPT; ++i) rb[(sub * TPT + i) * kOpLanes + row] = r[i];  // kShare: slot = sub
        }
        // one decision for all epilogue threads (the flag may change meanwhile)
        if (named_sync_or(kBarEpi, kEpiThreads, *abort_flag != 0u)) {
          run = false;
          break;
        }
        for (int e = ep; !kWriteX && e < p.IPT * NT; e += kEpiThreads) {
          const int nl = e / NT, jj = e % NT;
          const long long nn = (long long)rt * p.IPT + nl;
          const int j = tp * NT + jj;
          if (nn < p.N_A && j < p.N_B) {
            const float4* rb = res + (size_t)(tile & 1) * C::RES * kOpLanes + jj * kOpLanes + nl * p.T;
            float bv = -INFINITY, m = -INFINITY, s = 0.0f;
            int ba = 0;
            for (int tt = 0; tt < p.T; ++tt) {
              float4 e = rb[tt];
              if constexpr (C::kShare) {  // the two halves of the pair's angles (interleaved m)
                const float4 e1 = rb[kOpLanes + tt];
                if (e1.x > e.x || (e1.x == e.x && __float_as_int(e1.y) < __float_as_int(e.y))) {
                  e.x = e1.x;
                  e.y = e1.y;
                }
                if (p.lse_on) lse_merge(e.z, e.w, e1.z, e1.w);
              }
              if (e.x > bv) {
                bv = e.x;
                ba = tt * Q + __float_as_int(e.y);
              }
              if (p.lse_on) lse_merge(m, s, e.z, e.w);
            }
            const long long o = nn * p.N_B + j;
            p.best[o] = 6.283185307179586f * bv;
            p.arg[o] = ba;
            if (p.lse_on) p.lse[o] = m + logf(s);
          }
        }
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, kTmemCols);
  }
}

template <int Q>
int launch_tc(TcParams& p, bool write_x, const OperandLayout& La, int precision, cudaStream_t stream) {
  using C = TcCfg<Q>;
  const int planes = operand_planes(precision);
  p.split = is_split_precision(precision) ? 1 : 0;
  p.K = La.K;
  p.KC = La.KC;
  constexpr int NSPL = C::NSPL;
  p.KS = La.K / 16 / NSPL;
  p.Hp = La.Hp;
  p.IPT = La.IPT;
  p.nRT = (int)La.tiles;
  p.nTP = (p.N_B + C::NT - 1) / C::NT;
  p.idesc = idesc_f16((precision == RSVD_FP16 || precision == RSVD_FP16X3) ? 0u : 1u, 128, 16);
  p.a_bytes = (uint32_t)(kOpLanes * La.K * 2 / NSPL);
  p.b_bytes = (uint32_t)(16 * La.K * 2 / NSPL);
  const uint32_t dense_bytes = (uint32_t)(planes * C::NT * kOpGroups * La.K * 2);  // per producer warp
  p.dense_bytes = dense_bytes;
  const uint32_t res_bytes = 2u * C::RES * kOpLanes * 16u;
  const uint32_t kMaxSmem = 227u * 1024u;
  // Preferred layouts, first that fits: template blocks resident per unit
  // (single-pass forms) with two producers, then one producer; else the blocks
  // are rebuilt in every stage, two producers while three stages fit, else one.
  const uint32_t bres_bytes = (uint32_t)kOpGroups * p.b_bytes;
  struct Opt { int bres, nprod, min_stages; };
  const Opt opts[] = {{1, 2, 3}, {1, 1, 3}, {0, 2, 3}, {0, 1, 2}};
  bool found = false;
  for (const Opt& o : opts) {
    if (o.bres && (planes != 1 || NSPL != 1)) continue;
    const uint32_t sb = (uint32_t)((planes * (p.a_bytes + (o.bres ? 0u : p.b_bytes)) + 1023) / 1024 * 1024);
    const uint32_t fx = (uint32_t)o.nprod * dense_bytes + (o.bres ? bres_bytes : 0u) + res_bytes + 1024u;
    if (fx < kMaxSmem && (int)((kMaxSmem - fx) / sb) >= o.min_stages) {
      p.bres = o.bres;
      p.nprod = o.nprod;
      p.stage_bytes = sb;
      found = true;
      break;
    }
  }
  if (!found) return RSVD_EUNSUPPORTED;
  const uint32_t fixed = (uint32_t)p.nprod * dense_bytes + (p.bres ? bres_bytes : 0u) + res_bytes + 1024u;
  int stages = (int)((kMaxSmem - fixed) / p.stage_bytes);
  if (stages > 6) stages = 6;
  uint32_t smem = 0;
  // with two parts per group the stage count is even, so every stage always
  // holds the same part and its template block keeps one zero pattern
  for (; stages >= 2; stages -= (NSPL == 2 && (stages & 1) == 0) ? 2 : 1) {
    if (NSPL == 2 && (stages & 1)) continue;
    p.stages = stages;
    p.dense_off = (uint32_t)stages * p.stage_bytes;
    p.bres_off = p.dense_off + (uint32_t)p.nprod * dense_bytes;
    p.res_off = p.bres_off + (p.bres ? bres_bytes : 0u);
    p.bar_off = p.res_off + res_bytes;
    smem = p.bar_off + (uint32_t)(2 * stages + 3) * 8u + 8u;
    if (smem < 120u * 1024u) smem = 120u * 1024u;  // one CTA (and one TMEM allocation) per SM
    // the allocation also spans the operand descriptors read with their two
    // byte offsets exchanged (a 16-row-group stride of 2 KB from the last A block)
    const uint32_t last_a = (uint32_t)(stages - 1) * p.stage_bytes + (uint32_t)(planes - 1) * p.a_bytes;
    const uint32_t reach = last_a + (uint32_t)(p.KS - 1) * 4096u + 16u * 2048u + 256u;
    if (smem < reach) smem = reach;
    if (smem <= kMaxSmem) break;
  }
  if (stages < 2) return RSVD_EUNSUPPORTED;

  for (int k = 0; k < Q / 2; ++k) {
    const double aq = 2.0 * M_PI * k / Q, am = 2.0 * M_PI * k / (Q / 2);
    p.WQ[k] = make_float2((float)cos(aq), (float)-sin(aq));
    p.WM[k] = make_float2((float)cos(am), (float)-sin(am));
  }

  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return RSVD_ECUDA;
  const long long tiles = (long long)p.nRT * p.nTP;
  long long ch = tiles / ((long long)sms * 8);
  if (ch < 1) ch = 1;
  if (ch > 16) ch = 16;
  p.CH = (int)ch;
  const long long units = (long long)((p.nRT + p.CH - 1) / p.CH) * p.nTP;
  if (units > INT32_MAX) return RSVD_EUNSUPPORTED;
  p.nUnits = (int)units;
  const int grid = (int)(units < sms ? units : sms);

  const bool pair = p.bres && !p.split;
  auto kern = write_x ? (pair ? tc_align_kernel<Q, true, true> : tc_align_kernel<Q, true, false>)
                      : (pair ? tc_align_kernel<Q, false, true> : tc_align_kernel<Q, false, false>);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RSVD_ECUDA;
  kern<<<grid, kTcThreads, smem, stream>>>(p);
  return launch_status();
}

}  // namespace

// Shared entry of rsvd_align_best / rsvd_align_scores for the operand forms.
RSVD_HIDDEN int align_tc(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int precision,
                         float inv_sigma2, float* best, int32_t* arg, float* lse, float* X, cudaStream_t stream) {
  OperandLayout La{}, Lb{};
  if (!is_operand_precision(precision)) return RSVD_EUNSUPPORTED;
  if (!make_operand_layout(N_A, T, H, Q, &La) || !make_operand_layout(N_B, 1, H, Q, &Lb)) return RSVD_EUNSUPPORTED;
  TcParams p{};
  p.a = static_cast<const uint16_t*>(cA);
  p.b = static_cast<const uint16_t*>(cB);
  p.a_plane = La.plane_elems;
  p.b_plane = Lb.plane_elems;
  if (precision == RSVD_FP16X3) {
    p.sA = reinterpret_cast<const float*>(static_cast<const unsigned char*>(cA) + operand_scale_offset(La, precision));
    p.sB = reinterpret_cast<const float*>(static_cast<const unsigned char*>(cB) + operand_scale_offset(Lb, precision));
  }
  p.best = best;
  p.arg = arg;
  p.lse = lse;
  p.X = X;
  p.status = status_word();
  p.N_A = N_A;
  p.T = T;
  p.N_B = N_B;
  p.lse_on = lse ? 1 : 0;
  p.inv_sigma2 = inv_sigma2;
  if (Q == 128) return launch_tc<128>(p, X != nullptr, La, precision, stream);
  if (Q == 256) return launch_tc<256>(p, X != nullptr, La, precision, stream);
  return launch_tc<512>(p, X != nullptr, La, precision, stream);
}

}  // namespace rsvd
