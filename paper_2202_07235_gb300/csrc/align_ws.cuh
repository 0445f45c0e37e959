// Warp-specialised fused scoring kernel (rsvd_align_best, FP32, Q = 256 and 512).
//
// Same arithmetic as fused_align_kernel (eq. image_innerproduct_pm Steps 1-2,
// section 2.7 argmax, section 2.6 log-sum-exp), with the two phases running
// concurrently in different warps instead of alternating behind CTA-wide
// barriers:
// * contraction warps (CT threads = GC row groups x S angular slots) hold RT
//   image rows per slot in registers and write the half spectra of RP x TB
//   (row, template) pairs into one of two spectrum buffers;
// * FFT warps (FT threads, P2 lanes per pair) take a full buffer, run the C2R
//   FFT and the max/argmax/log-sum-exp of each pair, release the buffer, and
//   merge the rows of each image into the outputs.
// Hand-offs use named barriers (FULL[i]: contraction -> FFT, FREE[i]: FFT ->
// contraction). Templates arrive by bulk asynchronous copies (TMA) issued by
// one contraction thread into a double buffer, completing on mbarriers whose
// waits are bounded by a clock budget (a timeout is recorded in the status
// word and the CTA finishes without further copies).
#pragma once

#include "align_fused.cuh"
#include "ptx_sync.cuh"

namespace rsvd {

// S = 128: 256 contraction + 256 FFT threads, 3 image rows per thread (H <= 12);
// a batch of TB templates is one bulk copy.
// S = 256: 256 contraction threads keep 4 image rows x HP components each in
// registers and 256 FFT threads (16 lanes per pair) take 16 pairs per batch,
// i.e. TB = 4 templates. One template at H = 16 takes 32 KB of shared memory,
// so a batch arrives as SUB = 2 copies of TBL = 2 templates through a double
// buffer. The 512-thread block starts at 128 registers per thread; the
// contraction warps raise theirs to 168 and the FFT warps lower theirs to 88
// (setmaxnreg; 256 x 168 + 256 x 88 = the block's 65,536).
template <int S, int HP>
struct WsCfg {
  static constexpr int P1 = FftSplit<S>::P1, P2 = FftSplit<S>::P2, F = P2, RR = P1 / P2;
  static constexpr bool kWide = S >= 256;
  static constexpr int RT = kWide ? cmax(1, cmin(4, 64 / HP)) : cmax(1, cmin(4, 36 / HP));  // rows per thread
  static constexpr int GC = cmax(1, 256 / S);            // contraction row groups
  static constexpr int CT = GC * S;                      // contraction threads
  static constexpr int FT = 256;                         // FFT threads
  static constexpr int NT = CT + FT;
  static constexpr int RP = GC * RT;                     // rows per pass
  static constexpr int PGF = FT / F;                     // pairs per FFT round
  static constexpr int XP = P2 + 1;
  static constexpr int SP = pair_stride(S, P1, P2);
  static constexpr int PER_TB = 2 * HP * S * 8 + 2 * RP * SP * 8 + 24 * RP;
  static constexpr int TB_SMEM = (200 * 1024 - 2 * S * 8 - 64) / PER_TB;
  // templates per batch (FFT hand-off); per bulk copy (TBL, SUB copies per batch)
  static constexpr int TB = kWide ? cmax(1, PGF / RP) : cmax(1, cmin(TB_SMEM, cmax(1, PGF / RP)));
  static constexpr int TBL_SMEM = (224 * 1024 - 2 * S * 8 - 64 - 2 * TB * RP * SP * 8 - 24 * RP * TB) /
                                  (2 * HP * S * 8);
  static constexpr int TBL = kWide ? (TBL_SMEM >= TB ? TB : TBL_SMEM >= TB / 2 ? TB / 2 : 1) : TB;
  static constexpr int SUB = TB / TBL;
  static constexpr int PAIRS = RP * TB;
  static constexpr int SPB = PAIRS + (PGF - PAIRS % PGF) % PGF;  // pair regions per buffer (incl. dummies)
  static constexpr size_t SMEM = (size_t)2 * TBL * HP * S * 8 + (size_t)2 * SPB * SP * 8 + (size_t)2 * S * 8 +
                                 (size_t)2 * 3 * PAIRS * 4 + 64;
  // register split between the roles (kWide): 256 x (kRegC + kRegF) = 65,536
  static constexpr bool kRegSplit = kWide;
  static constexpr int kRegC = 168, kRegF = 88;
  static constexpr bool kFits = SMEM <= 227 * 1024 && S <= 256 && TBL >= 1 && TB % TBL == 0 &&
                                (!kRegSplit || (CT == 256 && FT == 256));
};

// clock budget of one bounded wait (about half a second at 2 GHz)
constexpr long long kWaitBudget = 1ll << 30;

enum : int { kBarCW = 1, kBarFW = 2, kBarFull0 = 3, kBarFree0 = 5 };

template <int S, int HP>
__global__ void __launch_bounds__(WsCfg<S, HP>::NT, 1) ws_align_kernel(const __grid_constant__ FusedParams p) {
  using C = WsCfg<S, HP>;
  constexpr int M = S, Q = 2 * S, P1 = C::P1, P2 = C::P2, RP = C::RP, RT = C::RT, TB = C::TB;
  constexpr int CT = C::CT, FT = C::FT, NT = C::NT, SP = C::SP, XP = C::XP, F = C::F, RR = C::RR;
  constexpr int PAIRS = C::PAIRS, PGF = C::PGF, TBL = C::TBL, SUB = C::SUB;
  static_assert(P1 * P2 == M && P1 % P2 == 0 && 32 % F == 0, "bad FFT split");

  extern __shared__ __align__(128) unsigned char ws_smem[];
  float2* tbuf = reinterpret_cast<float2*>(ws_smem);   // [2][TBL][HP][S], rows h >= H zero
  float2* spec = tbuf + 2 * TBL * HP * S;              // [2][SPB][SP] (PAIRS pairs + dummy regions)
  float2* twQ = spec + 2 * C::SPB * SP;                 // [M]
  float2* tw1 = twQ + M;                               // [M]
  float* res = reinterpret_cast<float*>(tw1 + M);      // [2][3][PAIRS]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(res + 2 * 3 * PAIRS);  // [2]
  int* abort_flag = reinterpret_cast<int*>(mbar + 2);

  const int tid = threadIdx.x;
  // CTAs that run at the same time share one chunk of templates (sized to stay
  // in L2): image group and template chunk of this CTA
  const int H = p.H, T = p.T;
  const int grp_id = p.ngroups > 0 ? (int)(blockIdx.x % (unsigned)p.ngroups) : (int)blockIdx.x;
  const int jc0 = p.ngroups > 0 ? (int)(blockIdx.x / (unsigned)p.ngroups) * p.jchunk : 0;
  const int N_B = p.ngroups > 0 ? min(p.jchunk, p.N_B - jc0) : p.N_B;  // templates of this CTA
  const float2* cB = p.cB + (size_t)jc0 * H * S;
  const int img0 = grp_id * p.IMG;
  if (img0 >= p.N_A) return;
  const int nimg = min(p.IMG, p.N_A - img0);
  const int rows_cta = nimg * T;
  const size_t row0 = (size_t)img0 * T;
  const bool want_lse = (p.lse != nullptr);
  const float two_pi = 6.28318530717958647692f;

  for (int i = tid; i < M; i += NT) {
    float sn, cs;
    sincospif(-2.0f * (float)i / (float)Q, &sn, &cs);
    twQ[i] = make_float2(cs, sn);
    const int k1 = i / P2, t = i % P2;
    sincospif(-2.0f * (float)(t * k1) / (float)M, &sn, &cs);
    tw1[i] = make_float2(cs, sn);
  }
  for (int i = tid; i < 2 * TBL * (HP - H) * S; i += NT) {
    const int slot = i / ((HP - H) * S), rem = i % ((HP - H) * S);
    tbuf[(size_t)slot * HP * S + (size_t)H * S + rem] = make_float2(0.f, 0.f);
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();

  const int nbatch = (N_B + TB - 1) / TB;
  const int passes = (rows_cta + RP - 1) / RP;
  const int total = passes * nbatch;
  // template copies: TBL templates each, nsubp per pass (the last batch of a
  // pass may need fewer than SUB); copy L holds templates (L % nsubp) * TBL + ..
  const int nsubp = (N_B + TBL - 1) / TBL;
  const long long total_loads = (long long)passes * nsubp;

  if (tid < CT) {
    // ======================= contraction warps =======================
    if constexpr (C::kRegSplit) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(C::kRegC));
    const int g = tid / S, s = tid % S;
    const bool slot0 = (s == 0);
    auto issue = [&](long long L) {
      const int j0 = (int)(L % nsubp) * TBL;
      const int nb = min(TBL, N_B - j0);
      const int buf = (int)(L & 1);
      const uint32_t per = (uint32_t)H * S * 8;
      mbar_arrive_expect_tx(&mbar[buf], per * nb);
      if (HP == H) {
        bulk_g2s(tbuf + (size_t)buf * TBL * HP * S, cB + (size_t)j0 * H * S, per * nb, &mbar[buf]);
      } else {
        for (int jj = 0; jj < nb; ++jj)
          bulk_g2s(tbuf + (size_t)(buf * TBL + jj) * HP * S, cB + (size_t)(j0 + jj) * H * S, per, &mbar[buf]);
      }
    };
    if (tid == 0) {
      if (total_loads > 0) issue(0);
      if (total_loads > 1) issue(1);
    }
    long long waited_upto = -1;  // copies this thread has seen complete
    long long issued_upto = total_loads < 2 ? total_loads - 1 : 1;
    float2 a[RT][HP];
    for (int it = 0; it < total; ++it) {
      const int pass = it / nbatch;
      const int ps = pass * RP;
      const int b = it % nbatch;
      if (b == 0) {
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
      }
      if (it >= 2) named_sync(kBarFree0 + (it & 1), CT + FT);
      float2* sp = spec + (size_t)(it & 1) * C::SPB * SP;
#pragma unroll 1
      for (int u = 0; u < SUB; ++u) {
        const int jb = b * TB + u * TBL;  // first template of this copy
        if (jb >= N_B) break;
        const long long L = (long long)pass * nsubp + b * SUB + u;
        const int nb = min(TBL, N_B - jb);
        if (*reinterpret_cast<volatile int*>(abort_flag) == 0) {
          if (mbar_wait_bounded(&mbar[L & 1], (uint32_t)((L >> 1) & 1), kWaitBudget)) {
            waited_upto = L;
          } else {
            record(p.status, kDevTimeout);
            atomicExch(abort_flag, 1);
          }
        }
        const float2* tb = tbuf + (size_t)(L & 1) * TBL * HP * S + s;
#pragma unroll 1
        for (int jj = 0; jj < TBL; ++jj) {
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
#pragma unroll
            for (int i = 0; i < RT; ++i) {
              const float re = slot0 ? PQ[i].x : PQ[i].x + PQ[i].y;
              const float im = slot0 ? PQ[i].y : RS[i].x - RS[i].y;
              sp[((g * RT + i) * TB + u * TBL + jj) * SP + s] = make_float2(re, im);
            }
          }
        }
        // every contraction thread is done with copy L's buffer: refill it with copy L + 2
        named_sync(kBarCW, CT);
        if (tid == 0 && L + 2 < total_loads && *reinterpret_cast<volatile int*>(abort_flag) == 0) {
          issue(L + 2);
          issued_upto = L + 2;
        }
      }
      named_arrive(kBarFull0 + (it & 1), CT + FT);
    }
    // copies issued but not waited for (only after a timeout): wait, bounded
    if (tid == 0) {
      for (long long L = waited_upto + 1; L <= issued_upto; ++L)
        (void)mbar_wait_bounded(&mbar[L & 1], (uint32_t)((L >> 1) & 1), kWaitBudget);
    }
  } else {
    // =========================== FFT warps ===========================
    if constexpr (C::kRegSplit) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(C::kRegF));
    const int ftid = tid - CT;
    const int ft = ftid % F;
    const float s2 = p.inv_sigma2;
    const float log2e = 1.44269504088896340736f;
    // merge items of a batch ((image, template) pairs) live on the first FFT
    // warp's lanes: only that warp pays their issue slots
    const int my_item = ftid;
    // at most (images touched by a pass) x TB items per batch; other threads skip the merge
    const bool merger = my_item < ((RP + T - 1) / T + 1) * TB;
    struct MergeSlot {
      int it, item;
      bool active, rmw, fetched;
      float ov, ol;
      int oi;
    };
    auto fetch = [&](MergeSlot& m, size_t o) {
      m.ov = p.best[o];
      m.oi = p.arg[o];
      m.ol = want_lse ? p.lse[o] : 0.f;
      m.fetched = true;
    };
    auto merge_prepare = [&](int it) {
      MergeSlot m{};
      m.it = it;
      m.item = my_item;
      const int ps = (it / nbatch) * RP;
      const int j0 = (it % nbatch) * TB;
      const int nb = min(TB, N_B - j0);
      const int il0 = ps / T;
      const int il1 = min(nimg - 1, (ps + RP - 1) / T);
      const int nitems = (il1 - il0 + 1) * nb;
      m.active = my_item < nitems;
      m.rmw = false;
      if (m.active) {
        const int il = il0 + my_item / nb, jj = my_item % nb;
        if (il * T < ps) {  // an earlier pass stored smaller t of this image
          m.rmw = true;
          // with several batches per pass that store was committed at least one
          // FULL sync ago, so it can be fetched now; with one batch it is
          // committed in this same iteration by another thread: fetch at commit
          if (nbatch >= 2) fetch(m, (size_t)(img0 + il) * p.N_B + jc0 + j0 + jj);
        }
      }
      return m;
    };
    auto merge_commit = [&](MergeSlot& m, const float* rs) {
      if (!m.active) return;
      const int ps = (m.it / nbatch) * RP;
      const int j0 = (m.it % nbatch) * TB;
      const int nb = min(TB, N_B - j0);
      const int il = ps / T + m.item / nb, jj = m.item % nb;
      const float* rv = rs;
      const int* ri = reinterpret_cast<const int*>(rs + PAIRS);
      const float* rlse = rs + 2 * PAIRS;
      const int rlo = max(il * T - ps, 0), rhi = min((il + 1) * T - ps, RP);
      float vb = -INFINITY, mm = -INFINITY, sm = 0.f;
      int ib = 0x7fffffff;
      for (int r_ = rlo; r_ < rhi; ++r_) {
        const int pr = r_ * TB + jj;
        const int t = ps + r_ - il * T;
        const float v = rv[pr];
        if (v > vb || r_ == rlo) {  // increasing t: ties keep the earlier index
          vb = v;
          ib = t * Q + ri[pr];
        }
        if (want_lse) lse_merge(mm, sm, rlse[pr], 1.0f);
      }
      const size_t o = (size_t)(img0 + il) * p.N_B + jc0 + j0 + jj;
      if (m.rmw) {
        if (!m.fetched) fetch(m, o);
        if (!(vb > m.ov)) {
          vb = m.ov;
          ib = m.oi;
        }
        if (want_lse) lse_merge(mm, sm, m.ol, 1.0f);
      }
      p.best[o] = vb;
      p.arg[o] = ib;
      if (want_lse) p.lse[o] = mm + logf(sm);
    };
    // Merge of batch `it` happens in iteration it+1, right after the FULL sync
    // (all FFT threads are then past batch it); its read-modify-write operands
    // are prefetched into registers one iteration earlier.
    MergeSlot ms;
    for (int it = 0; it < total; ++it) {
      const int ps = (it / nbatch) * RP;
      const int b = it % nbatch;
      const int j0 = b * TB;
      const int nb = min(TB, N_B - j0);
      named_sync(kBarFull0 + (it & 1), CT + FT);
      if (merger) {
        if (it > 0) merge_commit(ms, res + ((it - 1) & 1) * 3 * PAIRS);
        ms = merge_prepare(it);
      }
      float* rs = res + (it & 1) * 3 * PAIRS;
      const float2* specb = spec + (size_t)(it & 1) * C::SPB * SP;
#pragma unroll 1
      for (int pb = 0; pb < PAIRS; pb += PGF) {
        const int pr = pb + ftid / F;
        const int rl = pr / TB, jj = pr % TB;
        const bool ok = (pr < PAIRS) && (jj < nb) && (ps + rl < rows_cta);
        // groups without a pair (pr >= PAIRS) run on their own dummy region
        // (pr < SPB), keeping control flow uniform
        float2* sp = const_cast<float2*>(specb) + (size_t)pr * SP;
        float2 z[P1];
#pragma unroll
        for (int q1 = 0; q1 < P1; ++q1) {
          const int k = ft + P2 * q1;
          float2 A = sp[k];
          float2 B = cconj(sp[M - k]);
          if (q1 == 0) {  // k = 0 on lane 0: slot 0 packs the real X_hat(0), X_hat(Q/2)
            const bool k0 = (ft == 0);
            const float2 v = A;
            A = k0 ? make_float2(v.x, 0.f) : A;
            B = k0 ? make_float2(v.y, 0.f) : B;
          }
          const float2 d = cmul(csub(A, B), twQ[k]);
          z[q1] = make_float2(A.x + B.x - d.y, A.y + B.y + d.x);
        }
        RegDft<P1>::run(z);
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) z[k1] = cmul(z[k1], tw1[k1 * P2 + ft]);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < P1; ++k1) sp[k1 * XP + ft] = z[k1];
        __syncwarp();
        float2 y[RR][P2];
#pragma unroll
        for (int i = 0; i < RR; ++i) {
#pragma unroll
          for (int tp = 0; tp < P2; ++tp) y[i][tp] = sp[(ft * RR + i) * XP + tp];
          RegDft<P2>::run(y[i]);
        }
        // outputs in increasing m: m = 2 (ft*RR + i + P1*k2) + e at leaf (k2*RR + i)*2 + e
        float vals[2 * P1];
#pragma unroll
        for (int k2 = 0; k2 < P2; ++k2)
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            vals[(k2 * RR + i) * 2] = y[i][k2].x;
            vals[(k2 * RR + i) * 2 + 1] = y[i][k2].y;
          }
        float bv;
        int bj;
        tree_argmax<2 * P1>(vals, bv, bj);
        int bm = 2 * (ft * RR + (bj >> 1) % RR + P1 * ((bj >> 1) / RR)) + (bj & 1);
        if (!ok) {
          bv = -INFINITY;
          bm = 0x7fffffff;
        }
        argmax_warp_reduce(bv, bm, F);
        float lsev = 0.f;
        if (want_lse) {
          const float c = s2 * log2e, off = -c * bv;
#pragma unroll
          for (int t = 0; t < 2 * P1; ++t) vals[t] = exp2f(fmaf(c, vals[t], off));
          float sum = ok ? tree_sum<2 * P1>(vals) : 0.f;
#pragma unroll
          for (int o = F / 2; o >= 1; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, F);
          lsev = s2 * bv + logf(sum);
        }
        if (ok && ft == 0) {
          rs[pr] = bv;
          reinterpret_cast<int*>(rs + PAIRS)[pr] = bm;
          rs[2 * PAIRS + pr] = lsev;
        }
      }
      if (it + 2 < total) named_arrive(kBarFree0 + (it & 1), CT + FT);
    }
    if (total > 0) {
      named_sync(kBarFW, FT);  // every pair of the last batch is reduced
      if (merger) merge_commit(ms, res + ((total - 1) & 1) * 3 * PAIRS);
    }
  }
}

template <int S, int HP>
int launch_ws_cfg(const FusedParams& p0, cudaStream_t stream) {
  using C = WsCfg<S, HP>;
  if constexpr (!C::kFits) {
    return RSVD_EUNSUPPORTED;
  } else {
    FusedParams p = p0;
    p.IMG = images_per_cta(C::RP, p.T);
    const long long groups = ((long long)p.N_A + p.IMG - 1) / p.IMG;
    // template chunks of at most 40 MB (L2 holds one chunk while the image
    // groups running at the same time stream it), a multiple of TB templates
    const long long tbytes = (long long)p.N_B * p.H * S * 8;
    const long long kChunkBytes = 40ll << 20;
    int nchunk = (int)((tbytes + kChunkBytes - 1) / kChunkBytes);
    int jchunk = (p.N_B + nchunk - 1) / nchunk;
    jchunk = (jchunk + C::TB - 1) / C::TB * C::TB;
    nchunk = (p.N_B + jchunk - 1) / jchunk;
    p.ngroups = (int)groups;
    p.jchunk = jchunk;
    const long long grid = groups * nchunk;
    if (groups > 0x7fffffffLL || grid > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
    if (cudaFuncSetAttribute(ws_align_kernel<S, HP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM) !=
        cudaSuccess)
      return RSVD_ECUDA;
    ws_align_kernel<S, HP><<<(unsigned)grid, C::NT, C::SMEM, stream>>>(p);
    return launch_status();
  }
}

RSVD_HIDDEN int launch_ws_s128(int HP, const FusedParams& p, cudaStream_t stream);
RSVD_HIDDEN int launch_ws_s256(int HP, const FusedParams& p, cudaStream_t stream);

}  // namespace rsvd
