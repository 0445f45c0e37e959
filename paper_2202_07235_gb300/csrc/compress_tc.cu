// Compression with the projection on the tensor cores (rsvd_compress, FP32
// output, Q in {256, 512}, H <= 16, R <= 128).
//
// Section 3.2 (principal-image-rings), with the translation T_delta of
// section 5 and the section 2.3 discrete Fourier-Bessel coefficients:
//   A_t(r, psi) = A(k_r, psi) exp(-i k_r (dx_t cos psi + dy_t sin psi))
//   a_t(h, psi) = sum_r W[r][h] A_t(r, psi),  W[r][h] = U[r][h] sqrt(w_r)
//   a_t(h, q)   = (1/Q) sum_psi a_t(h, psi) e^{-2 pi i q psi / Q}
// The projection is, for each object, translation and block of 64 angles, a
// real GEMM D[128 x 16] = A[128 x R] W[R x 16] with rows (angle, re | im) and
// columns h: tcgen05 MMAs of kind::tf32 accumulating in TMEM. FP32 accuracy
// comes from splitting both operands into TF32 hi + lo parts and summing
// A_hi W_hi + A_hi W_lo + A_lo W_hi (each part keeps 11 significand bits, so
// the dropped A_lo W_lo term and the rounding of the parts are about 2^-22 of
// each product).
//
// One CTA (256 threads) per object:
// * the half rings of a block of 64 angles (psi < Q/2; the other half is the
//   conjugate for real images) are staged in shared memory, R x 64 complex;
// * for each translation and each half of the ring range, eight warps build
//   the A operand (phase multiply, TF32 split) into one of two stage buffers
//   while the tensor core works on the other; a ninth warp issues the 24 MMAs
//   of each stage (one elected lane) and commits them to the buffer's
//   mbarrier (full / empty barriers per buffer, a tile barrier per group of
//   translations, a read-back barrier before the columns are reused);
// * per block of angles the translations' results (16 TMEM columns each, up
//   to 32 translations per pass) are read back and written, as a_t(h, psi),
//   into the rows of the output that will hold a_t(h, q);
// * a last pass runs the Q-point transform of each (t, h) row in place (16
//   lanes per row: P1-point DFTs in registers, twiddles, an exchange through
//   shared memory, 16-point DFTs) and writes the slots as compress_kernel.
// Every wait is clock-bounded; a timeout is recorded in the status word.
#include <math.h>

#include "compress_tc.cuh"
#include "tc_ptx.cuh"

namespace rsvd {
namespace {

constexpr int kCtWorkers = 256;               // builders / read-back / transform (8 warps)
constexpr int kCtThreads = kCtWorkers + 32;   // + the MMA warp
constexpr int kCtPsi = 64;          // angles per block (128 operand rows: re, im)
constexpr int kCtMaxT = 32;         // translations per TMEM pass (16 columns each)
constexpr long long kCtBudget = 1LL << 31;

template <int Q>
struct CtSplit;
template <>
struct CtSplit<256> {
  static constexpr int P1 = 16, P2 = 16;
};
template <>
struct CtSplit<512> {
  static constexpr int P1 = 32, P2 = 16;
};

struct CtLayout {
  int Rp;           // rings rounded up to a multiple of 32 (zero rings past R)
  int KS;           // K-steps of 8 per stage (half of Rp)
  uint32_t a_plane; // bytes of one plane of a stage's A operand: 128 rows x Rp/2
  uint32_t w_plane; // bytes of one half of the W operand: 16 rows x Rp
  // the transform pass reuses [0, xbytes) (staged rings and operands) as its
  // exchange buffers; twiddles and barriers sit above both
  uint32_t off_img, off_w, off_a, off_tw, off_bar, smem;
  uint32_t tcols;   // TMEM columns allocated
};

template <int Q>
inline CtLayout ct_layout(int R) {
  constexpr int P1 = CtSplit<Q>::P1, P2 = CtSplit<Q>::P2;
  CtLayout L{};
  L.Rp = (R + 31) / 32 * 32;
  L.KS = L.Rp / 16;
  L.a_plane = 128u * (uint32_t)(L.Rp / 2) * 4u;
  L.w_plane = 16u * (uint32_t)L.Rp * 4u;
  L.off_img = 0;
  L.off_w = L.off_img + (uint32_t)L.Rp * kCtPsi * 8u;
  L.off_a = (L.off_w + 2u * L.w_plane + 1023u) / 1024u * 1024u;
  const uint32_t end_a = L.off_a + 2u * 2u * L.a_plane;  // 2 stage buffers x (hi, lo)
  const uint32_t xbytes = (uint32_t)(kCtWorkers / P2) * P1 * (P2 + 1) * 8u;
  L.off_tw = ((end_a > xbytes ? end_a : xbytes) + 15u) / 16u * 16u;
  L.off_bar = L.off_tw + (uint32_t)(P1 * P2) * 8u;
  L.smem = L.off_bar + 64u;
  return L;
}

__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ bool ct_wait(uint64_t* bar, uint32_t parity, int* status, volatile int* abort_flag) {
  if (*abort_flag) return false;
  if (mbar_wait_bounded(bar, parity, kCtBudget)) return true;
  record(status, kDevTimeout);
  *abort_flag = 1;
  return false;
}


template <int Q>
__global__ void __launch_bounds__(kCtThreads, 1) compress_tc_kernel(const __grid_constant__ CompressTcParams p,
                                                                    const CtLayout L) {
  constexpr int M = Q / 2, NCHUNK = M / kCtPsi;
  constexpr int P1 = CtSplit<Q>::P1, P2 = CtSplit<Q>::P2, XP = P2 + 1, RR = P1 / P2;
  static_assert(P2 == 16 && P1 % P2 == 0 && P1 * P2 == Q, "bad transform split");
  extern __shared__ __align__(1024) unsigned char ct_smem[];
  float2* img = reinterpret_cast<float2*>(ct_smem + L.off_img);         // [Rp][64]
  uint32_t* wop = reinterpret_cast<uint32_t*>(ct_smem + L.off_w);        // [2 planes][Rp/4][16][4]
  unsigned char* aop = ct_smem + L.off_a;                                 // [2 bufs][2 planes][Rp/8][128][4]
  float2* tw = reinterpret_cast<float2*>(ct_smem + L.off_tw);            // [P1][P2] W_Q^{t k1}
  uint64_t* full = reinterpret_cast<uint64_t*>(ct_smem + L.off_bar);     // [2] operand built (8 warps)
  uint64_t* empty = full + 2;                                            // [2] the stage's MMAs done
  uint64_t* tile = empty + 2;                                            // a group's MMAs done
  uint64_t* tfree = tile + 1;                                            // TMEM read back (8 warps)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfree + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = blockIdx.x;
  const int R = p.R, H = p.H, T = p.T, Rp = L.Rp;
  const int RB = Rp / 8;  // rings per builder thread and stage (a multiple of 4)
  constexpr int kMmaWarp = kCtWorkers / 32;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], kCtWorkers / 32);
      mbar_init(&empty[i], 1);
    }
    mbar_init(tile, 1);
    mbar_init(tfree, kCtWorkers / 32);
    *abort_flag = 0;
    fence_mbar_init();
  }
  // W = U sqrt(w) as TF32 hi and lo planes, K-major B operand (row h, column r)
  for (int i = tid; i < Rp * 16; i += kCtThreads) {
    const int r = i >> 4, h = i & 15;
    const float w = (r < R && h < H) ? (float)p.U[r * H + h] * p.sw[r] : 0.0f;
    const float hi = tf32_rn(w), lo = tf32_rn(w - hi);
    const int idx = ((r >> 2) * 16 + h) * 4 + (r & 3);
    wop[idx] = __float_as_uint(hi);
    wop[Rp * 16 + idx] = __float_as_uint(lo);
  }
  for (int i = tid; i < P1 * P2; i += kCtThreads) {
    const int k1 = i / P2, t = i % P2;
    float sn, cs;
    sincospif(-2.0f * (float)(t * k1) / (float)Q, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
  fence_proxy_async_smem();
  if (warp == kMmaWarp) {
    tmem_alloc(tmem_slot, L.tcols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const float2* src = p.polar + (size_t)n * R * Q;

  if (warp == kMmaWarp) {
    // ================= MMA issue (converged warp, one elected lane) =================
    const uint32_t leader = elect_one();
    const uint32_t idesc = idesc_f16(2u, 128, 16);  // kind::tf32, M = 128, N = 16
    const uint32_t a_lbo = 128u * 16u, b_lbo = 16u * 16u, sbo = 128u;
    const uint64_t a_step = (2u * a_lbo) >> 4, b_step = (2u * b_lbo) >> 4;
    const uint32_t w_hi = smem_addr(wop), w_lo = w_hi + L.w_plane;
    long long stage = 0, groups = 0;
    for (int c = 0; c < NCHUNK; ++c) {
      for (int t0 = 0; t0 < T; t0 += kCtMaxT) {
        const int tg = min(kCtMaxT, T - t0);
        // the previous group's columns have been read back
        if (groups > 0) (void)ct_wait(tfree, (uint32_t)((groups - 1) & 1), p.status, abort_flag);
        tc_fence_after();
        for (int tl = 0; tl < tg; ++tl) {
          for (int kh = 0; kh < 2; ++kh, ++stage) {
            const int b = (int)(stage & 1);
            (void)ct_wait(&full[b], (uint32_t)((stage >> 1) & 1), p.status, abort_flag);
            tc_fence_after();
            const uint32_t ahi = smem_addr(aop + (size_t)b * 2u * L.a_plane), alo = ahi + L.a_plane;
            const uint32_t koff = (uint32_t)(kh * (Rp / 8)) * 256u;
            const uint64_t ad = smem_desc_kmajor(ahi, a_lbo, sbo), al = smem_desc_kmajor(alo, a_lbo, sbo);
            const uint64_t bd = smem_desc_kmajor(w_hi + koff, b_lbo, sbo), bl = smem_desc_kmajor(w_lo + koff, b_lbo, sbo);
            const uint32_t d = tmem_base + (uint32_t)(tl * 16);
            if (!*abort_flag) {
              for (int ks = 0; ks < L.KS; ++ks) {
                tc_mma_tf32_by(leader, d, ad + ks * a_step, bd + ks * b_step, idesc, (kh > 0 || ks > 0) ? 1u : 0u);
                tc_mma_tf32_by(leader, d, ad + ks * a_step, bl + ks * b_step, idesc, 1u);
                tc_mma_tf32_by(leader, d, al + ks * a_step, bd + ks * b_step, idesc, 1u);
              }
            }
            tc_commit_by(leader, &empty[b]);  // the stage buffer may be rebuilt
            __syncwarp();
          }
        }
        tc_commit_by(leader, tile);  // the group's columns are complete
        __syncwarp();
        ++groups;
      }
    }
  } else {
    // ============ operand builders, read-back and transform (8 warps) ============
    const int psl = (warp & 1) * 32 + lane;  // 32 consecutive angles per warp
    const int rb = warp >> 1;                // a quarter of the stage's rings
    long long stage = 0, groups = 0;
    for (int c = 0; c < NCHUNK; ++c) {
      // ---- stage the half rings of this block of 64 angles ----
      // (no stage buffer or staged ring is in use: the previous block's
      // groups have all been read back, so their MMAs are complete)
      named_sync(1, kCtWorkers);
#pragma unroll 8
      for (int i = tid; i < Rp * kCtPsi; i += kCtWorkers) {
        const int r = i / kCtPsi, ps = i % kCtPsi;
        img[i] = (r < R) ? src[(size_t)r * Q + c * kCtPsi + ps] : make_float2(0.f, 0.f);
      }
      named_sync(1, kCtWorkers);
      const int psi = c * kCtPsi + psl;
      float spsi, cpsi;
      sincospif(2.0f * (float)psi / (float)Q, &spsi, &cpsi);
      for (int t0 = 0; t0 < T; t0 += kCtMaxT) {
        const int tg = min(kCtMaxT, T - t0);
        for (int tl = 0; tl < tg; ++tl) {
          const int t = t0 + tl;
          const float rho = p.dx[t] * cpsi + p.dy[t] * spsi;
          float2 step = make_float2(1.f, 0.f);
          if (p.uniform) {
            float sn, cs;
            sincosf(p.dk * rho, &sn, &cs);
            step = make_float2(cs, -sn);
          }
          for (int kh = 0; kh < 2; ++kh, ++stage) {
            const int b = (int)(stage & 1);
            const long long use = stage >> 1;
            if (use > 0) (void)ct_wait(&empty[b], (uint32_t)((use - 1) & 1), p.status, abort_flag);
            // ---- A operand of (t, kh): rows (angle, re | im), columns = rings ----
            unsigned char* ahi = aop + (size_t)b * 2u * L.a_plane;
            unsigned char* alo = ahi + L.a_plane;
            const int r0 = kh * (Rp / 2) + rb * RB;
            float2 ph = make_float2(1.f, 0.f);
            for (int j0 = 0; j0 < RB; j0 += 4) {
              float vr[4], vi[4];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                const int r = r0 + j0 + jj;
                if (!p.uniform || (j0 + jj) == 0 || (r & 7) == 0) {
                  float sn, cs;
                  sincosf(p.k[r < R ? r : R - 1] * rho, &sn, &cs);
                  ph = make_float2(cs, -sn);
                } else {
                  ph = cmul(ph, step);
                }
                const float2 u = (r < R) ? cmul(img[r * kCtPsi + psl], ph) : make_float2(0.f, 0.f);
                vr[jj] = u.x;
                vi[jj] = u.y;
              }
              float hr[4], lr[4], hm[4], lm[4];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                hr[jj] = tf32_rn(vr[jj]);
                lr[jj] = tf32_rn(vr[jj] - hr[jj]);
                hm[jj] = tf32_rn(vi[jj]);
                lm[jj] = tf32_rn(vi[jj] - hm[jj]);
              }
              const int kg = (rb * RB + j0) >> 2;  // K group of 4 within the stage
              // row psl: real part, row 64 + psl: imaginary part (consecutive
              // lanes write consecutive 16-byte rows)
              const uint32_t o_re = ((uint32_t)kg * 128u + (uint32_t)psl) * 16u, o_im = o_re + 64u * 16u;
              *reinterpret_cast<float4*>(ahi + o_re) = make_float4(hr[0], hr[1], hr[2], hr[3]);
              *reinterpret_cast<float4*>(alo + o_re) = make_float4(lr[0], lr[1], lr[2], lr[3]);
              *reinterpret_cast<float4*>(ahi + o_im) = make_float4(hm[0], hm[1], hm[2], hm[3]);
              *reinterpret_cast<float4*>(alo + o_im) = make_float4(lm[0], lm[1], lm[2], lm[3]);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[b]);
          }
        }
        // ---- the group's results: a_t(h, psi) into the output rows ----
        (void)ct_wait(tile, (uint32_t)(groups & 1), p.status, abort_flag);
        __syncwarp();
        tc_fence_after();
        {
          const int qd = warp & 3, half = warp >> 2;
          const int row = qd * 32 + lane;  // real parts in rows 0..63, imaginary parts in 64..127
          const int ps = c * kCtPsi + (row & 63), comp = row >> 6;
          for (int tl = half; tl < tg; tl += 2) {
            uint32_t r[16];
            tmem_ld16_issue(tmem_base + ((uint32_t)(qd * 32) << 16) + (uint32_t)(tl * 16), r);
            tmem_wait_ld_tie<16>(r);
            float* o = reinterpret_cast<float*>(p.out + ((size_t)n * T + t0 + tl) * H * M + ps) + comp;
#pragma unroll
            for (int h = 0; h < 16; ++h)
              if (h < H) o[(size_t)h * M * 2] = __uint_as_float(r[h]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tfree);
        ++groups;
      }
    }

    // ---- the Q-point transform of every (t, h) row, in place ----
    named_sync(1, kCtWorkers);  // every group read back: the operand area is free
    {
      float2* xb = reinterpret_cast<float2*>(ct_smem);  // [16 rows][P1][XP]
      const int ft = tid % P2, rs = tid / P2;
      const float invQ = 1.0f / (float)Q;
      float2* x = xb + (size_t)rs * P1 * XP;
      for (int base = 0; base < T * H; base += kCtWorkers / P2) {
        const int idx = base + rs;
        const bool valid = idx < T * H;
        float2* row = p.out + ((size_t)n * T + (valid ? idx / H : 0)) * H * M + (size_t)(valid ? idx % H : 0) * M;
        float2 z[P1];
#pragma unroll
        for (int q1 = 0; q1 < P1 / 2; ++q1) {
          const float2 v = valid ? row[ft + P2 * q1] : make_float2(0.f, 0.f);
          z[q1] = v;
          z[q1 + P1 / 2] = cconj(v);  // a(psi + Q/2) = conj a(psi)
        }
        RegDft<P1>::run(z);
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) z[k1] = cmul(z[k1], tw[k1 * P2 + ft]);
        __syncwarp();
#pragma unroll
        for (int k1 = 0; k1 < P1; ++k1) x[k1 * XP + ft] = z[k1];
        __syncwarp();
        if (valid) {
#pragma unroll
          for (int i = 0; i < RR; ++i) {
            const int k1 = ft * RR + i;
            float2 y[P2];
#pragma unroll
            for (int q2 = 0; q2 < P2; ++q2) y[q2] = x[k1 * XP + q2];
            RegDft<P2>::run(y);
            // X(k1 + P1 k2); slots q = 1 .. M-1, slot 0 = (Re X(0), Re X(M))
#pragma unroll
            for (int k2 = 0; k2 < P2 / 2; ++k2) {
              const int q = k1 + P1 * k2;
              if (q == 0) {
                row[0] = make_float2(y[0].x * invQ, y[P2 / 2].x * invQ);
              } else {
                row[q] = make_float2(y[k2].x * invQ, y[k2].y * invQ);
              }
            }
          }
        }
        __syncwarp();
      }
    }
  }

  // every MMA has completed (the builders waited for the last group, or the
  // waits gave up after a timeout and the drain below bounds the rest)
  if (warp == kMmaWarp) {
    const uint32_t leader = elect_one();
    tc_commit_by(leader, tile);
    __syncwarp();
    long long groups = (long long)NCHUNK * ((T + kCtMaxT - 1) / kCtMaxT);
    (void)mbar_wait_bounded(tile, (uint32_t)(groups & 1), kCtBudget);
  }
  __syncthreads();
  if (warp == kMmaWarp) {
    tc_fence_after();
    tmem_dealloc(tmem_base, L.tcols);
  }
}

template <int Q>
int launch_q(const CompressTcParams& p, cudaStream_t stream) {
  CtLayout L = ct_layout<Q>(p.R);
  if (L.smem > 227u * 1024u) return RSVD_EUNSUPPORTED;
  // one CTA (and one 512-column TMEM allocation) per SM
  L.tcols = 512;
  if (L.smem < 120u * 1024u) L.smem = 120u * 1024u;
  if (cudaFuncSetAttribute(compress_tc_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem) !=
      cudaSuccess)
    return RSVD_ECUDA;
  compress_tc_kernel<Q><<<p.N, kCtThreads, L.smem, stream>>>(p, L);
  return launch_status();
}

}  // namespace

RSVD_HIDDEN int launch_compress_tc(const CompressTcParams& p, cudaStream_t stream) {
  if (p.R < 1 || p.R > 128 || p.H < 1 || p.H > 16 || p.T < 1 || p.T > kMaxT || p.N < 1) return RSVD_EUNSUPPORTED;
  if (p.Q == 256) return launch_q<256>(p, stream);
  if (p.Q == 512) return launch_q<512>(p, stream);
  return RSVD_EUNSUPPORTED;
}

}  // namespace rsvd
