// Volume alignment (section 4): volumes given by spherical-harmonic
// coefficients A_l^m(k_r) on R shells (complex64 [N][R][L+1][2L+1], m + L in the
// last index, zero for |m| > l), rotations tau = (gamma, beta, alpha),
// X(tau) = <A, R_tau B>, with R_tau = R_z(alpha) R_y(beta) R_z(gamma) acting on
// the coefficients through e^{-i m1 alpha} d^l_{m1 m2}(beta) e^{-i m2 gamma}.
//
// * vol_kernel_C / vol_kernel_D (FP64): the radial kernel of eq.
//   Volume_simple_radial_kern (sqrt(w_r w_r') weights, l = 0 excluded) and the
//   degree kernel of eq. Volume_simple_degree_kern (rows and columns l = 0 zero),
//   averaged over the targets; their principal vectors by the Jacobi solver.
// * vol_tables_kernel (FP64 recursion): [v_d^T d]_{m1 m2}(beta_b) = sum_l V_{l d} d^l_{m1 m2}(beta_b)
//   (eq. principal_degree_wigner), by the three-term recursion in l from the
//   closed form of d^{l0}, l0 = max(|m1|, |m2|).
// * vol_compress_kernel: principal-volume-shells [u_h^T A]_l^m = sum_r U_rh sqrt(w_r) A_l^m(k_r).
// * vol_align_kernel: one CTA per (volume, target): Steps 1 and 1b of eq.
//   volume_innerproduct_pm into registers (Hermitian part, each thread owns a
//   few (m1, m2) and their mirrors), then per pair of interior angles Step 2
//   and one packed complex 2-D DFT of Step 3 (zero-padded to Mp x Mp), and a
//   running max / argmax over (beta, alpha, gamma).
#include <math.h>

#include <algorithm>
#include <cstdlib>
#include <type_traits>

#include "align_common.cuh"

namespace rsvd {

RSVD_HIDDEN int launch_jacobi(const double* C, double* A, double* V, int R, int H, double* U, double* eig, int batch,
                              cudaStream_t st);

namespace {

constexpr int kVolMaxL = 31;
constexpr int kVolMaxHD = 8;
constexpr int kVolMaxHC = 16;
constexpr int kAlignThreads = 512;

struct VolKernParams {
  const float2* B;  // [N_B][R][L+1][M]
  double* out;
  int N_B, R, L;
  double w[kMaxR];
};

__global__ void vol_kernel_C(const __grid_constant__ VolKernParams p) {
  const float2* B = p.B;
  const int N_B = p.N_B, R = p.R, L = p.L;
  const double* w = p.w;
  double* C = p.out;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= R * R) return;
  const int r = i / R, s = i % R, M = 2 * L + 1;
  double acc = 0.0;
  for (int j = 0; j < N_B; ++j) {
    const float2* br = B + ((size_t)j * R + r) * (L + 1) * M;
    const float2* bs = B + ((size_t)j * R + s) * (L + 1) * M;
    for (int l = 1; l <= L; ++l)
      for (int m = L - l; m <= L + l; ++m) {
        const float2 x = br[l * M + m], y = bs[l * M + m];
        acc += (double)x.x * y.x + (double)x.y * y.y;
      }
  }
  C[i] = acc * sqrt(w[r] * w[s]) / N_B;
}

__global__ void vol_kernel_D(const __grid_constant__ VolKernParams p) {
  const float2* B = p.B;
  const int N_B = p.N_B, R = p.R, L = p.L;
  const double* w = p.w;
  double* D = p.out;
  const int L1 = L + 1;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L1 * L1) return;
  const int l = i / L1, k = i % L1, M = 2 * L + 1;
  double acc = 0.0;
  if (l > 0 && k > 0) {
    const int mm = min(l, k);
    for (int j = 0; j < N_B; ++j)
      for (int r = 0; r < R; ++r) {
        const float2* b = B + ((size_t)j * R + r) * L1 * M;
        double s = 0.0;
        for (int m = L - mm; m <= L + mm; ++m) {
          const float2 x = b[l * M + m], y = b[k * M + m];
          s += (double)x.x * y.x + (double)x.y * y.y;
        }
        acc += w[r] * s;
      }
  }
  D[i] = acc / N_B;
}

// d^l_{l, m}(beta) = (-1)^{l-m} sqrt(binom(2l, l+m)) cos(beta/2)^{l+m} sin(beta/2)^{l-m}
__device__ double d_top(int l, int m, double c, double s) {
  const double lb = 0.5 * (lgamma(2.0 * l + 1.0) - lgamma((double)(l + m) + 1.0) - lgamma((double)(l - m) + 1.0));
  const double v = exp(lb) * pow(c, (double)(l + m)) * pow(s, (double)(l - m));
  return ((l - m) & 1) ? -v : v;
}

// thread per (beta_b, m1, m2): T[b][m1+L][m2+L][d] = sum_l V[l][d] d^l_{m1 m2}(beta_b)
constexpr int kVolMaxBeta = 256;

struct VolTableParams {
  const double* V;  // dev [L+1][HD]
  float* T;         // dev [n_beta][M][M][kVolMaxHD], zero for d >= HD
  int n_beta, L, HD;
  double betas[kVolMaxBeta];
};

__global__ void vol_tables_kernel(const __grid_constant__ VolTableParams p) {
  const double* V = p.V;
  const double* betas = p.betas;
  const int n_beta = p.n_beta, L = p.L, HD = p.HD;
  float* T = p.T;
  const int M = 2 * L + 1;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n_beta * M * M) return;
  const int b = (int)(i / (M * M)), e = (int)(i % (M * M));
  const int m1 = e / M - L, m2 = e % M - L;
  const double beta = betas[b];
  const double c = cos(0.5 * beta), s = sin(0.5 * beta), cb = cos(beta);
  const int l0 = max(abs(m1), abs(m2));
  double d;
  if (m1 == l0) d = d_top(l0, m2, c, s);
  else if (m1 == -l0) d = (((l0 + m2) & 1) ? -1.0 : 1.0) * d_top(l0, -m2, c, s);
  else if (m2 == l0) d = (((l0 - m1) & 1) ? -1.0 : 1.0) * d_top(l0, m1, c, s);
  else d = d_top(l0, -m1, c, s);
  double acc[kVolMaxHD];
#pragma unroll
  for (int q = 0; q < kVolMaxHD; ++q) acc[q] = (q < HD) ? V[l0 * HD + q] * d : 0.0;
  double dm1 = 0.0;
  int l = l0;
  if (l0 == 0 && L >= 1) {  // d^1_{00} = cos beta starts the recursion
    dm1 = d;
    d = cb;
    l = 1;
#pragma unroll
    for (int q = 0; q < kVolMaxHD; ++q)
      if (q < HD) acc[q] += V[1 * HD + q] * d;
  }
  for (; l < L; ++l) {
    const double a = (l + 1.0) * (2.0 * l + 1.0) /
                     sqrt(((l + 1.0) * (l + 1.0) - (double)m1 * m1) * ((l + 1.0) * (l + 1.0) - (double)m2 * m2));
    const double nxt = a * ((cb - (double)m1 * m2 / (l * (l + 1.0))) * d -
                            sqrt(((double)l * l - (double)m1 * m1) * ((double)l * l - (double)m2 * m2)) /
                                (l * (2.0 * l + 1.0)) * dm1);
    dm1 = d;
    d = nxt;
#pragma unroll
    for (int q = 0; q < kVolMaxHD; ++q)
      if (q < HD) acc[q] += V[(l + 1) * HD + q] * d;
  }
  float4* out = reinterpret_cast<float4*>(T + ((size_t)b * M * M + e) * kVolMaxHD);
  out[0] = make_float4((float)acc[0], (float)acc[1], (float)acc[2], (float)acc[3]);
  out[1] = make_float4((float)acc[4], (float)acc[5], (float)acc[6], (float)acc[7]);
}

struct VolCompressParams {
  const float2* A;  // [N][R][L+1][M]
  float2* out;      // [N][HC][L+1][M]
  const double* U;  // dev [R][HC]
  int N, R, L, HC;
  double sw[kMaxR];
};

// thread per (volume, l, m): HCT >= HC accumulators (HC rounded up to 4)
template <int HCT>
__global__ void __launch_bounds__(256) vol_compress_kernel(const __grid_constant__ VolCompressParams p) {
  __shared__ float uw_s[kMaxR * HCT];  // U[r][h] sqrt(w_r)
  for (int i = threadIdx.x; i < p.R * HCT; i += blockDim.x) {
    const int r = i / HCT, h = i % HCT;
    uw_s[i] = (h < p.HC) ? (float)(p.U[r * p.HC + h] * p.sw[r]) : 0.f;
  }
  __syncthreads();
  const int M = 2 * p.L + 1, LM = (p.L + 1) * M;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)p.N * LM) return;
  const int n = (int)(i / LM), lm = (int)(i % LM);
  const int l = lm / M, m = lm % M - p.L;
  float2 acc[HCT];
#pragma unroll
  for (int h = 0; h < HCT; ++h) acc[h] = make_float2(0.f, 0.f);
  if (abs(m) <= l) {
    const float2* a = p.A + (size_t)n * p.R * LM + lm;
#pragma unroll 4
    for (int r = 0; r < p.R; ++r) {
      const float2 x = __ldcs(a + (size_t)r * LM);  // streamed once
      const float* u = uw_s + r * HCT;
#pragma unroll
      for (int h = 0; h < HCT; ++h) {
        acc[h].x = fmaf(u[h], x.x, acc[h].x);
        acc[h].y = fmaf(u[h], x.y, acc[h].y);
      }
    }
  }
  float2* out = p.out + (size_t)n * p.HC * LM + lm;
#pragma unroll
  for (int h = 0; h < HCT; ++h)
    if (h < p.HC) out[(size_t)h * LM] = acc[h];
}

struct VolAlignParams {
  const float2* cA;  // [N_A][HC][L+1][M]
  const float2* cB;  // [N_B][HC][L+1][M]
  const float* T;    // [n_beta][M][M][kVolMaxHD]
  float* best;
  int32_t* arg;
  const double* V;   // dev [L+1][HD]
  int N_A, N_B, HC, L, HD, n_beta;
  // chunk[w * kVolMaxEPT + q]: the 32-entry chunk of the (m1, m2) half grid that
  // warp w holds in slot q (see vol_chunk_plan)
  uint8_t chunk[16 * 4];
};

constexpr int kVolMaxEPT = 4;

// Entry of the (m1, m2) half grid (e = (m1 + L) M + m2 + L < (M^2 + 1) / 2) that
// thread tid holds in slot q; entries past the half grid are unused slots.
__device__ __forceinline__ int vol_entry(const VolAlignParams& p, int tid, int q) {
  return (int)p.chunk[(tid >> 5) * kVolMaxEPT + q] * 32 + (tid & 31);
}


// Forward 8-point DFT (kernel e^{-2 pi i n k / 8}) in place, natural order in
// and out: even/odd split into two 4-point DFTs and one butterfly layer.
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  constexpr float kR = 0.70710678118654752f;  // 1 / sqrt(2)
  float2 e[4], o[4];
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // h = 0: x0 x2 x4 x6; h = 1: x1 x3 x5 x7
    const float2 a0 = x[h], a1 = x[h + 2], a2 = x[h + 4], a3 = x[h + 6];
    const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y), d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
    const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y), d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
    float2* r = h ? o : e;
    r[0] = make_float2(s02.x + s13.x, s02.y + s13.y);
    r[2] = make_float2(s02.x - s13.x, s02.y - s13.y);
    r[1] = make_float2(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
    r[3] = make_float2(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
  }
  // W8^k o[k]: W8 = (1 - i)/sqrt 2, W8^2 = -i, W8^3 = -(1 + i)/sqrt 2
  const float2 t1 = make_float2(kR * (o[1].x + o[1].y), kR * (o[1].y - o[1].x));
  const float2 t2 = make_float2(o[2].y, -o[2].x);
  const float2 t3 = make_float2(kR * (o[3].y - o[3].x), -kR * (o[3].x + o[3].y));
  x[0] = make_float2(e[0].x + o[0].x, e[0].y + o[0].y);
  x[4] = make_float2(e[0].x - o[0].x, e[0].y - o[0].y);
  x[1] = make_float2(e[1].x + t1.x, e[1].y + t1.y);
  x[5] = make_float2(e[1].x - t1.x, e[1].y - t1.y);
  x[2] = make_float2(e[2].x + t2.x, e[2].y + t2.y);
  x[6] = make_float2(e[2].x - t2.x, e[2].y - t2.y);
  x[3] = make_float2(e[3].x + t3.x, e[3].y + t3.y);
  x[7] = make_float2(e[3].x - t3.x, e[3].y - t3.y);
}

// Shared-memory layout of vol_align_kernel. Region 0 holds the compressed
// pair (Step 1) and is then reused by the transform buffers.
struct VolSmem {
  size_t region0, tw, vs, red, total;
};

constexpr int kS = 65;  // row stride (complex values) of the 64 x 64 transform buffers

__host__ __device__ inline VolSmem vol_align_layout(int HC, int L, int Mp) {
  const size_t M = 2 * L + 1;
  const size_t pair = 2 * (size_t)HC * (L + 1) * M * sizeof(float2);
  const size_t ept = ((M * M + 1) / 2 + kAlignThreads - 1) / kAlignThreads;
  // Mp = 64: the zero-padded input grid and the work grid [64][kS] each, and the
  // prefetched Wigner-table entries of one pair of angles [ept][2][threads][8]
  const size_t fft = Mp == 64 ? 2 * 64 * kS * sizeof(float2) + ept * 2 * kAlignThreads * kVolMaxHD * sizeof(float)
                              : (size_t)Mp * (Mp + 1) * sizeof(float2);
  VolSmem s;
  s.region0 = ((pair > fft ? pair : fft) + 15) & ~(size_t)15;
  s.tw = s.region0;
  s.vs = s.tw + 64 * sizeof(float2);
  s.red = s.vs + (((size_t)(L + 1) * kVolMaxHD * sizeof(float) + 15) & ~(size_t)15);
  s.total = s.red + 32 * sizeof(float) + 32 * sizeof(int);
  return s;
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit_all() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Running max over eight scores visited in increasing flat index
// base + f * step (f = 0..7): ties keep the earliest.
__device__ __forceinline__ void best8(const float (&v)[8], int base, int step, float& bv, int& bi) {
  float m = v[0];
#pragma unroll
  for (int f = 1; f < 8; ++f) m = fmaxf(m, v[f]);
  if (m > bv) {
    int f = 7;
#pragma unroll
    for (int g = 6; g >= 0; --g)
      if (v[g] == m) f = g;
    bv = m;
    bi = base + f * step;
  }
}

// One CTA per (volume n, target j), 512 threads.
//  Steps 1 + 1b: thread owns EPT entries e of the first half of the M x M
//    (m1, m2) grid together with their mirrors -m; it accumulates the
//    Hermitian part Yh_d(m) = (Y_d(m) + (-1)^{m1-m2} conj Y_d(-m)) / 2, where
//    Y_d = sum_l V_{l d} sum_h conj(a_{h,l}^{m1}) b_{h,l}^{m2}. Because
//    [v_d^T d](-m) = (-1)^{m1-m2} [v_d^T d](m), Step 2 applied to Yh gives a
//    Hermitian Xhat whose 2-D transform is Re X, for any input coefficients.
//  Per pair of interior angles (b1, b2): Step 2 forms Xhat(b1) + i Xhat(b2) at m
//    and its mirror, one complex 2-D transform gives X(b1) in the real part and
//    X(b2) in the imaginary part (Step 3), and each thread keeps a running
//    max / argmax; one block reduction at the end.
//  Mp = 64: rows then columns, each as two radix-8 passes in registers over a
//    [64][65] grid (line = thread mod 64); the next pair's table entries are
//    fetched asynchronously into per-thread slots during the transform.
//  Mp = 16, 32: radix-2 passes in shared memory on bit-reversed input.
// kReal: the volumes and targets are real (A_l^{-m} = (-1)^{l+m} conj A_l^m), so
// the mirror product equals (-1)^{m1-m2} conj of the direct one and the
// Hermitian part of Step 1b is the direct accumulation: half the Step-1 work.
template <int Mp, int EPT, bool kReal>
__global__ void __launch_bounds__(kAlignThreads) vol_align_kernel(const __grid_constant__ VolAlignParams p) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const int L = p.L, M = 2 * L + 1, LM = (L + 1) * M, HC = p.HC, MM = M * M, Mh = (MM + 1) / 2;
  const VolSmem lay = vol_align_layout(HC, L, Mp);
  float2* sa = reinterpret_cast<float2*>(vsm);  // [HC][L+1][M]
  float2* sb = sa + (size_t)HC * LM;            // [HC][L+1][M]
  float2* tw = reinterpret_cast<float2*>(vsm + lay.tw);
  float* Vs = reinterpret_cast<float*>(vsm + lay.vs);  // [L+1][kVolMaxHD]
  float* rv = reinterpret_cast<float*>(vsm + lay.red);
  int* ri = reinterpret_cast<int*>(rv + 32);
  const int n = blockIdx.x / p.N_B, j = blockIdx.x % p.N_B;
  const int tid = threadIdx.x;
  {
    const float2* ga = p.cA + (size_t)n * HC * LM;
    const float2* gb = p.cB + (size_t)j * HC * LM;
    for (int i = tid; i < HC * LM; i += kAlignThreads) {
      cp_async8(sa + i, ga + i);
      cp_async8(sb + i, gb + i);
    }
    cp_async_commit_all();
  }
  if (tid < 64) {
    float sn, cs;
    sincospif(-2.0f * (float)(Mp == 64 ? tid : (tid % (Mp / 2))) / (float)Mp, &sn, &cs);
    tw[tid] = make_float2(cs, sn);
  }
  for (int i = tid; i < (L + 1) * kVolMaxHD; i += kAlignThreads) {
    const int l = i / kVolMaxHD, d = i % kVolMaxHD;
    Vs[i] = (d < p.HD) ? (float)p.V[l * p.HD + d] : 0.f;
  }
  cp_async_wait_all();
  __syncthreads();

  // Steps 1 and 1b (Hermitian part)
  float2 Y[EPT][kVolMaxHD];
  const size_t hstride = (size_t)(L + 1) * M;
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
#pragma unroll
    for (int d = 0; d < kVolMaxHD; ++d) Y[q][d] = make_float2(0.f, 0.f);
    const int e = vol_entry(p, tid, q);
    const bool on = e < Mh;
    const int i1 = on ? e / M : 0, i2 = on ? e % M : 0;
    const int l0 = on ? max(abs(i1 - L), abs(i2 - L)) : L + 1;
    const int lstart = __reduce_min_sync(0xffffffffu, l0);
    const float s = ((i1 + i2) & 1) ? -0.5f : 0.5f;
    for (int l = lstart; l <= L; ++l) {
      if (l >= l0) {
        float2 x = make_float2(0.f, 0.f), y = make_float2(0.f, 0.f);
        const float2* ah = sa + l * M;
        const float2* bh = sb + l * M;
        for (int h = 0; h < HC; ++h, ah += hstride, bh += hstride) {
          const float2 a = ah[i1], b = bh[i2];
          x.x = fmaf(a.x, b.x, fmaf(a.y, b.y, x.x));
          x.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, x.y));
          if constexpr (!kReal) {
            const float2 a2 = ah[2 * L - i1], b2 = bh[2 * L - i2];
            y.x = fmaf(a2.x, b2.x, fmaf(a2.y, b2.y, y.x));
            y.y = fmaf(a2.x, b2.y, fmaf(-a2.y, b2.x, y.y));
          }
        }
        const float2 xh = kReal ? x : make_float2(fmaf(0.5f, x.x, s * y.x), fmaf(0.5f, x.y, -s * y.y));
        const float4 v0 = *reinterpret_cast<const float4*>(Vs + l * kVolMaxHD);
        const float4 v1 = *reinterpret_cast<const float4*>(Vs + l * kVolMaxHD + 4);
        const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int d = 0; d < kVolMaxHD; ++d) {
          Y[q][d].x = fmaf(vv[d], xh.x, Y[q][d].x);
          Y[q][d].y = fmaf(vv[d], xh.y, Y[q][d].y);
        }
      }
    }
  }
  __syncthreads();  // region 0 is reused below

  float bv = -INFINITY;
  int bidx = 0x7fffffff;
  constexpr int kMM = Mp * Mp;
  if constexpr (Mp == 64) {
    float2* xin = reinterpret_cast<float2*>(vsm);  // [64][kS]: Xhat at (m1 mod 64, m2 mod 64), zero elsewhere
    float2* wk = xin + 64 * kS;                     // [64][kS]
    float* Ts = reinterpret_cast<float*>(wk + 64 * kS);  // [EPT][2][threads][8]
    for (int i = tid; i < 64 * kS; i += kAlignThreads) xin[i] = make_float2(0.f, 0.f);
    __syncthreads();  // zeros before any thread writes its entries
    // grid offsets of this thread's entries and of their mirrors
    int off[EPT], offm[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = min(vol_entry(p, tid, q), Mh - 1);
      const int m1 = e / M - L, m2 = e % M - L;
      off[q] = ((m1 + 64) & 63) * kS + ((m2 + 64) & 63);
      offm[q] = ((64 - m1) & 63) * kS + ((64 - m2) & 63);
    }
    auto prefetch = [&](int b) {  // table entries of angles b and b + 1 (or b again)
      const float* T1 = p.T + (size_t)b * MM * kVolMaxHD;
      const float* T2 = b + 1 < p.n_beta ? T1 + (size_t)MM * kVolMaxHD : T1;
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = vol_entry(p, tid, q);
        if (e < Mh) {
          float* dst = Ts + ((q * 2) * kAlignThreads + tid) * kVolMaxHD;
          cp_async16(dst, T1 + (size_t)e * kVolMaxHD);
          cp_async16(dst + 4, T1 + (size_t)e * kVolMaxHD + 4);
          cp_async16(dst + kAlignThreads * kVolMaxHD, T2 + (size_t)e * kVolMaxHD);
          cp_async16(dst + kAlignThreads * kVolMaxHD + 4, T2 + (size_t)e * kVolMaxHD + 4);
        }
      }
      cp_async_commit_all();
    };
    prefetch(0);
    const int ln = tid & 63, jj = tid >> 6;  // line and radix-8 digit of this thread
    const bool row_on = (ln <= L) || (ln >= Mp - L);
    for (int b1 = 0; b1 < p.n_beta; b1 += 2) {
      const bool two = b1 + 1 < p.n_beta;
      cp_async_wait_all();  // own slots only: no barrier needed
      // Step 2 at m and -m
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = vol_entry(p, tid, q);
        if (e < Mh) {
          const float* t = Ts + ((q * 2) * kAlignThreads + tid) * kVolMaxHD;
          const float4 a0 = *reinterpret_cast<const float4*>(t), a1 = *reinterpret_cast<const float4*>(t + 4);
          const float4 c0 = *reinterpret_cast<const float4*>(t + kAlignThreads * kVolMaxHD);
          const float4 c1 = *reinterpret_cast<const float4*>(t + kAlignThreads * kVolMaxHD + 4);
          const float t1[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float t2[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
          float2 h1 = make_float2(0.f, 0.f), h2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int d = 0; d < kVolMaxHD; ++d) {
            h1.x = fmaf(t1[d], Y[q][d].x, h1.x);
            h1.y = fmaf(t1[d], Y[q][d].y, h1.y);
            h2.x = fmaf(t2[d], Y[q][d].x, h2.x);
            h2.y = fmaf(t2[d], Y[q][d].y, h2.y);
          }
          if (!two) h2 = make_float2(0.f, 0.f);
          xin[off[q]] = make_float2(h1.x - h2.y, h1.y + h2.x);
          xin[offm[q]] = make_float2(h1.x + h2.y, h2.x - h1.y);
        }
      }
      if (b1 + 2 < p.n_beta) prefetch(b1 + 2);  // lands during the transform
      __syncthreads();
      float2 x[8];
      // rows (transform over m2): n = jj + 8k, W64^{jj f2} twiddle, f = f2 + 8 f1
      if (row_on) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = xin[ln * kS + jj + 8 * k];
        dft8(x);
#pragma unroll
        for (int f = 1; f < 8; ++f) x[f] = cmul(x[f], tw[jj * f]);
#pragma unroll
        for (int f = 0; f < 8; ++f) wk[ln * kS + jj + 8 * f] = x[f];
      }
      __syncthreads();
      if (row_on) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = wk[ln * kS + k + 8 * jj];
        dft8(x);
        // frequency c = jj + 8 f stored at column position 8 jj + f (same set as read)
#pragma unroll
        for (int f = 0; f < 8; ++f) wk[ln * kS + 8 * jj + f] = x[f];
      }
      __syncthreads();
      // columns (transform over m1), one column position per thread line
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int r = jj + 8 * k;
        x[k] = (r <= L || r >= Mp - L) ? wk[r * kS + ln] : make_float2(0.f, 0.f);
      }
      dft8(x);
#pragma unroll
      for (int f = 1; f < 8; ++f) x[f] = cmul(x[f], tw[jj * f]);
#pragma unroll
      for (int f = 0; f < 8; ++f) wk[(jj + 8 * f) * kS + ln] = x[f];
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = wk[(k + 8 * jj) * kS + ln];
      dft8(x);
      // position ln = 8 f2 + f1 holds c = f2 + 8 f1; row a = jj + 8 f
      const int base = jj * Mp + (ln >> 3) + 8 * (ln & 7);
      {
        float v[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) v[f] = x[f].x;
        best8(v, b1 * kMM + base, 8 * Mp, bv, bidx);
      }
      if (two) {
        float v[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) v[f] = x[f].y;
        best8(v, (b1 + 1) * kMM + base, 8 * Mp, bv, bidx);
      }
      // no barrier needed here: the next Step 2 writes only xin (last read
      // before two barriers) and the next row pass writes wk after its barrier
    }
  } else {
    constexpr int lg = Mp == 32 ? 5 : 4;
    constexpr int XP = Mp + 1;
    float2* buf = reinterpret_cast<float2*>(vsm);  // [Mp][Mp+1]
    for (int b1 = 0; b1 < p.n_beta; b1 += 2) {
      const bool two = b1 + 1 < p.n_beta;
      const float* T1 = p.T + (size_t)b1 * MM * kVolMaxHD;
      const float* T2 = two ? T1 + (size_t)MM * kVolMaxHD : T1;
      for (int i = tid; i < Mp * XP; i += kAlignThreads) buf[i] = make_float2(0.f, 0.f);
      __syncthreads();
#pragma unroll
      for (int q = 0; q < EPT; ++q) {
        const int e = vol_entry(p, tid, q);
        if (e < Mh) {
          float2 h1 = make_float2(0.f, 0.f), h2 = make_float2(0.f, 0.f);
#pragma unroll
          for (int d = 0; d < kVolMaxHD; ++d) {
            const float t1 = __ldg(T1 + (size_t)e * kVolMaxHD + d), t2 = __ldg(T2 + (size_t)e * kVolMaxHD + d);
            h1.x = fmaf(t1, Y[q][d].x, h1.x);
            h1.y = fmaf(t1, Y[q][d].y, h1.y);
            h2.x = fmaf(t2, Y[q][d].x, h2.x);
            h2.y = fmaf(t2, Y[q][d].y, h2.y);
          }
          if (!two) h2 = make_float2(0.f, 0.f);
          const int m1 = e / M - L, m2 = e % M - L;
          const unsigned u1 = (unsigned)(m1 + Mp) & (Mp - 1), u2 = (unsigned)(m2 + Mp) & (Mp - 1);
          const unsigned v1 = (unsigned)(Mp - m1) & (Mp - 1), v2 = (unsigned)(Mp - m2) & (Mp - 1);
          buf[(__brev(u1) >> (32 - lg)) * XP + (__brev(u2) >> (32 - lg))] = make_float2(h1.x - h2.y, h1.y + h2.x);
          buf[(__brev(v1) >> (32 - lg)) * XP + (__brev(v2) >> (32 - lg))] = make_float2(h1.x + h2.y, h2.x - h1.y);
        }
      }
      __syncthreads();
#pragma unroll
      for (int dim = 0; dim < 2; ++dim) {
#pragma unroll
        for (int half = 1; half < Mp; half *= 2) {
          const int stride = Mp / (2 * half);
          for (int bf = tid; bf < Mp * Mp / 2; bf += kAlignThreads) {
            const int line = bf / (Mp / 2), k = bf % (Mp / 2);
            const int pos = k % half, grp = k / half;
            const int i0 = grp * 2 * half + pos, i1 = i0 + half;
            const int a0 = dim == 0 ? line * XP + i0 : i0 * XP + line;
            const int a1 = dim == 0 ? line * XP + i1 : i1 * XP + line;
            const float2 u = buf[a0];
            const float2 v = cmul(buf[a1], tw[pos * stride]);
            buf[a0] = make_float2(u.x + v.x, u.y + v.y);
            buf[a1] = make_float2(u.x - v.x, u.y - v.y);
          }
          __syncthreads();
        }
      }
      for (int i = tid; i < kMM; i += kAlignThreads) {
        const float v = buf[(i / Mp) * XP + (i % Mp)].x;
        if (v > bv) {
          bv = v;
          bidx = b1 * kMM + i;
        }
      }
      if (two)
        for (int i = tid; i < kMM; i += kAlignThreads) {
          const float v = buf[(i / Mp) * XP + (i % Mp)].y;
          if (v > bv) {
            bv = v;
            bidx = (b1 + 1) * kMM + i;
          }
        }
      __syncthreads();
    }
  }
  argmax_warp_reduce(bv, bidx, 32);
  if ((tid & 31) == 0) {
    rv[tid >> 5] = bv;
    ri[tid >> 5] = bidx;
  }
  __syncthreads();
  if (tid == 0) {
    float tb = rv[0];
    int ti = ri[0];
    for (int w_ = 1; w_ < kAlignThreads / 32; ++w_)
      if (rv[w_] > tb || (rv[w_] == tb && ri[w_] < ti)) {
        tb = rv[w_];
        ti = ri[w_];
      }
    p.best[(size_t)n * p.N_B + j] = tb;
    p.arg[(size_t)n * p.N_B + j] = ti == 0x7fffffff ? 0 : ti;
  }
}

}  // namespace
}  // namespace rsvd

extern "C" size_t rsvd_volume_build_workspace_bytes(int R, int L) {
  if (R <= 0 || R > rsvd::kMaxR || L < 1 || L > rsvd::kVolMaxL) return 0;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t a = up((size_t)R * R * sizeof(double)), b = up((size_t)(L + 1) * (L + 1) * sizeof(double));
  return 3 * a + 3 * b;
}

extern "C" int rsvd_build_volume_svd(int R, int L, const double* w, const void* targets, int N_B, int HC, int HD,
                                     double* U, double* eigU, double* V, double* eigV, void* workspace,
                                     size_t workspace_bytes, void* stream) {
  using namespace rsvd;
  if (!w || !targets || !U || !eigU || !V || !eigV || N_B <= 0) return RSVD_EINVAL;
  if (R <= 0 || L < 1 || HC <= 0 || HD <= 0 || HC > R || HD > L + 1) return RSVD_EINVAL;
  if (R > kMaxR || L > kVolMaxL) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)targets & 7u) || ((uintptr_t)U & 7u) || ((uintptr_t)V & 7u)) return RSVD_EINVAL;
  const size_t need = rsvd_volume_build_workspace_bytes(R, L);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255u)) return RSVD_EWORKSPACE;
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t a = up((size_t)R * R * sizeof(double)), b = up((size_t)(L + 1) * (L + 1) * sizeof(double));
  char* ws = static_cast<char*>(workspace);
  double* C = reinterpret_cast<double*>(ws);
  double* CA = reinterpret_cast<double*>(ws + a);
  double* CV = reinterpret_cast<double*>(ws + 2 * a);
  double* D = reinterpret_cast<double*>(ws + 3 * a);
  double* DA = reinterpret_cast<double*>(ws + 3 * a + b);
  double* DV = reinterpret_cast<double*>(ws + 3 * a + 2 * b);
  VolKernParams kp{};
  kp.B = static_cast<const float2*>(targets);
  kp.N_B = N_B;
  kp.R = R;
  kp.L = L;
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    kp.w[r] = w[r];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  kp.out = C;
  vol_kernel_C<<<(R * R + 127) / 128, 128, 0, st>>>(kp);
  int rc = launch_status();
  if (rc != RSVD_OK) return rc;
  kp.out = D;
  vol_kernel_D<<<((L + 1) * (L + 1) + 127) / 128, 128, 0, st>>>(kp);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  if ((rc = launch_jacobi(C, CA, CV, R, HC, U, eigU, 1, st)) != RSVD_OK) return rc;
  return launch_jacobi(D, DA, DV, L + 1, HD, V, eigV, 1, st);
}

extern "C" int rsvd_volume_tables(int L, int HD, const double* V, const double* betas, int n_beta, float* tables,
                                  void* stream) {
  using namespace rsvd;
  if (!V || !betas || !tables || L < 1 || HD <= 0 || n_beta <= 0) return RSVD_EINVAL;
  if ((uintptr_t)tables & 15u) return RSVD_EINVAL;
  if (L > kVolMaxL || HD > kVolMaxHD || HD > L + 1 || n_beta > kVolMaxBeta) return RSVD_EUNSUPPORTED;
  VolTableParams tp{};
  tp.V = V;
  tp.T = tables;
  tp.n_beta = n_beta;
  tp.L = L;
  tp.HD = HD;
  for (int b = 0; b < n_beta; ++b) {
    if (!isfinite(betas[b])) return RSVD_EINVAL;
    tp.betas[b] = betas[b];
  }
  const int M = 2 * L + 1;
  const long long total = (long long)n_beta * M * M;
  vol_tables_kernel<<<(unsigned)((total + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(tp);
  return launch_status();
}

extern "C" int rsvd_compress_volume(int R, int L, const double* w, const double* U, int HC, const void* volumes, int N,
                                    void* out, void* stream) {
  using namespace rsvd;
  if (!w || !U || !volumes || !out || R <= 0 || L < 1 || HC <= 0 || N <= 0 || HC > R) return RSVD_EINVAL;
  if (R > kMaxR || L > kVolMaxL || HC > kVolMaxHC) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)volumes & 7u) || ((uintptr_t)out & 7u) || ((uintptr_t)U & 7u)) return RSVD_EINVAL;
  VolCompressParams cp{};
  cp.A = static_cast<const float2*>(volumes);
  cp.out = static_cast<float2*>(out);
  cp.U = U;
  cp.N = N;
  cp.R = R;
  cp.L = L;
  cp.HC = HC;
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    cp.sw[r] = sqrt(w[r]);
  }
  const long long total = (long long)N * (L + 1) * (2 * L + 1);
  if ((total + 255) / 256 > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
  const unsigned grid = (unsigned)((total + 255) / 256);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (HC <= 4)
    vol_compress_kernel<4><<<grid, 256, 0, st>>>(cp);
  else if (HC <= 8)
    vol_compress_kernel<8><<<grid, 256, 0, st>>>(cp);
  else if (HC <= 12)
    vol_compress_kernel<12><<<grid, 256, 0, st>>>(cp);
  else
    vol_compress_kernel<16><<<grid, 256, 0, st>>>(cp);
  return launch_status();
}

namespace rsvd {
namespace {

// Step 1 of a (m1, m2) entry loops over l = max(|m1|, |m2|) .. L, and a warp runs
// as many iterations as its entry with the smallest l; the first half grid is
// cut into 32-entry chunks (one per warp and slot) and the chunks are dealt to
// the 16 warps, heaviest first, each to the warp with the least work so far
// that still has a free slot, so that no warp carries much more Step-1 work
// than the mean (at L = 24: 33 iterations for the busiest warp instead of 44).
void vol_chunk_plan(int L, int ept, uint8_t* chunk) {
  const int M = 2 * L + 1, Mh = (M * M + 1) / 2, warps = kAlignThreads / 32, n = warps * ept;
  int work[16 * kVolMaxEPT], order[16 * kVolMaxEPT], load[16] = {0}, used[16] = {0};
  for (int c = 0; c < n; ++c) {
    int lmin = L + 1;
    for (int e = 32 * c; e < 32 * c + 32 && e < Mh; ++e) {
      const int a = abs(e / M - L), b = abs(e % M - L);
      lmin = std::min(lmin, std::max(a, b));
    }
    work[c] = L + 1 - lmin;
    order[c] = c;
  }
  std::stable_sort(order, order + n, [&](int x, int y) { return work[x] > work[y]; });
  for (int i = 0; i < n; ++i) {
    int w = -1;
    for (int k = 0; k < warps; ++k)
      if (used[k] < ept && (w < 0 || load[k] < load[w])) w = k;
    chunk[w * kVolMaxEPT + used[w]++] = (uint8_t)order[i];
    load[w] += work[order[i]];
  }
}

int align_volumes_impl(bool real, const void* cA, int N_A, const void* cB, int N_B, int HC, int L, const double* V,
                       int HD, const float* tables, int n_beta, int Mp, float* best, int32_t* arg, void* stream) {
  if (!cA || !cB || !V || !tables || !best || !arg || N_A <= 0 || N_B <= 0 || HC <= 0 || L < 1 || HD <= 0 ||
      n_beta <= 0)
    return RSVD_EINVAL;
  if (L > kVolMaxL || HD > kVolMaxHD || HC > kVolMaxHC || HD > L + 1) return RSVD_EUNSUPPORTED;
  if (!(Mp == 16 || Mp == 32 || Mp == 64) || Mp < 2 * L + 1) return RSVD_EUNSUPPORTED;
  if ((long long)N_A * N_B > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)tables & 15u) || ((uintptr_t)cA & 7u) || ((uintptr_t)cB & 7u)) return RSVD_EINVAL;
  VolAlignParams ap{};
  ap.cA = static_cast<const float2*>(cA);
  ap.cB = static_cast<const float2*>(cB);
  ap.T = tables;
  ap.best = best;
  ap.arg = arg;
  ap.V = V;
  ap.N_A = N_A;
  ap.N_B = N_B;
  ap.HC = HC;
  ap.L = L;
  ap.HD = HD;
  ap.n_beta = n_beta;
  const int M = 2 * L + 1;
  const int ept = ((M * M + 1) / 2 + kAlignThreads - 1) / kAlignThreads;
  if (ept > kVolMaxEPT) return RSVD_EUNSUPPORTED;
  vol_chunk_plan(L, Mp == 64 ? ept : 1, ap.chunk);
  const size_t smem = vol_align_layout(HC, L, Mp).total;
  if (smem > 227 * 1024) return RSVD_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto go = [&](auto kern) -> int {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return RSVD_ECUDA;
    kern<<<(unsigned)((long long)N_A * N_B), kAlignThreads, smem, st>>>(ap);
    return launch_status();
  };
  auto pick = [&](auto real_tag) -> int {
    constexpr bool R_ = decltype(real_tag)::value;
    if (Mp == 16) return go(vol_align_kernel<16, 1, R_>);
    if (Mp == 32) return go(vol_align_kernel<32, 1, R_>);
    if (ept <= 1) return go(vol_align_kernel<64, 1, R_>);
    if (ept <= 2) return go(vol_align_kernel<64, 2, R_>);
    if (ept <= 3) return go(vol_align_kernel<64, 3, R_>);
    if (ept <= 4) return go(vol_align_kernel<64, 4, R_>);
    return (int)RSVD_EUNSUPPORTED;
  };
  return real ? pick(std::true_type{}) : pick(std::false_type{});
}
}  // namespace
}  // namespace rsvd

extern "C" int rsvd_align_volumes(const void* cA, int N_A, const void* cB, int N_B, int HC, int L, const double* V,
                                  int HD, const float* tables, int n_beta, int Mp, float* best, int32_t* arg,
                                  void* stream) {
  return rsvd::align_volumes_impl(false, cA, N_A, cB, N_B, HC, L, V, HD, tables, n_beta, Mp, best, arg, stream);
}

extern "C" int rsvd_align_volumes_real(const void* cA, int N_A, const void* cB, int N_B, int HC, int L,
                                       const double* V, int HD, const float* tables, int n_beta, int Mp, float* best,
                                       int32_t* arg, void* stream) {
  return rsvd::align_volumes_impl(true, cA, N_A, cB, N_B, HC, L, V, HD, tables, n_beta, Mp, best, arg, stream);
}
