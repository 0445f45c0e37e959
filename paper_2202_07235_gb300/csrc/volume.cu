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
//   volume_innerproduct_pm into registers (each thread owns a few (m1, m2)),
//   then per interior angle Step 2 and the 2-D DFT of Step 3 in shared memory
//   (zero-padded to Mp x Mp), and the max / argmax over (beta, alpha, gamma).
#include <math.h>

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

// thread per (beta_b, m1, m2): T[b][d][m1+L][m2+L] = sum_l V[l][d] d^l_{m1 m2}(beta_b)
constexpr int kVolMaxBeta = 256;

struct VolTableParams {
  const double* V;  // dev [L+1][HD]
  float* T;         // dev [n_beta][HD][M][M]
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
#pragma unroll
  for (int q = 0; q < kVolMaxHD; ++q)
    if (q < HD) T[((size_t)b * HD + q) * M * M + e] = (float)acc[q];
}

struct VolCompressParams {
  const float2* A;  // [N][R][L+1][M]
  float2* out;      // [N][HC][L+1][M]
  const double* U;  // dev [R][HC]
  int N, R, L, HC;
  double sw[kMaxR];
};

__global__ void vol_compress_kernel(const __grid_constant__ VolCompressParams p) {
  __shared__ float uw_s[kMaxR * kVolMaxHC];  // U[r][h] sqrt(w_r)
  for (int i = threadIdx.x; i < p.R * kVolMaxHC; i += blockDim.x) {
    const int r = i / kVolMaxHC, h = i % kVolMaxHC;
    uw_s[i] = (h < p.HC) ? (float)(p.U[r * p.HC + h] * p.sw[r]) : 0.f;
  }
  __syncthreads();
  const float* uw = uw_s;
  const int M = 2 * p.L + 1, LM = (p.L + 1) * M;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)p.N * LM) return;
  const int n = (int)(i / LM), lm = (int)(i % LM);
  const int l = lm / M, m = lm % M - p.L;
  float2 acc[kVolMaxHC];
#pragma unroll
  for (int h = 0; h < kVolMaxHC; ++h) acc[h] = make_float2(0.f, 0.f);
  if (abs(m) <= l) {
    for (int r = 0; r < p.R; ++r) {
      const float2 a = p.A[((size_t)n * p.R + r) * LM + lm];
#pragma unroll
      for (int h = 0; h < kVolMaxHC; ++h) {
        const float u = uw[r * kVolMaxHC + h];
        acc[h].x = fmaf(u, a.x, acc[h].x);
        acc[h].y = fmaf(u, a.y, acc[h].y);
      }
    }
  }
#pragma unroll
  for (int h = 0; h < kVolMaxHC; ++h)
    if (h < p.HC) p.out[((size_t)n * p.HC + h) * LM + lm] = acc[h];
}

struct VolAlignParams {
  const float2* cA;  // [N_A][HC][L+1][M]
  const float2* cB;  // [N_B][HC][L+1][M]
  const float* T;    // [n_beta][HD][M][M]
  float* best;
  int32_t* arg;
  const double* V;   // dev [L+1][HD]
  int N_A, N_B, HC, L, HD, n_beta, Mp, log2Mp;
};

template <int EPT>
__global__ void __launch_bounds__(kAlignThreads) vol_align_kernel(const __grid_constant__ VolAlignParams p) {
  extern __shared__ __align__(16) unsigned char vsm[];
  const int L = p.L, M = 2 * L + 1, LM = (L + 1) * M, HC = p.HC, HD = p.HD, Mp = p.Mp, XP = Mp + 1;
  float2* sa = reinterpret_cast<float2*>(vsm);   // [HC][L+1][M]
  float2* sb = sa + (size_t)HC * LM;             // [HC][L+1][M]
  float2* buf = sb + (size_t)HC * LM;            // [Mp][Mp + 1]
  float2* tw = buf + (size_t)Mp * XP;            // [Mp/2] W_Mp^k
  float* rv = reinterpret_cast<float*>(tw + Mp / 2);
  int* ri = reinterpret_cast<int*>(rv + 32);
  float* Vs = reinterpret_cast<float*>(ri + 32);  // [L+1][kVolMaxHD]
  const int n = blockIdx.x / p.N_B, j = blockIdx.x % p.N_B;
  const int tid = threadIdx.x;
  for (int i = tid; i < HC * LM; i += kAlignThreads) {
    sa[i] = p.cA[(size_t)n * HC * LM + i];
    sb[i] = p.cB[(size_t)j * HC * LM + i];
  }
  for (int i = tid; i < Mp / 2; i += kAlignThreads) {
    float sn, cs;
    sincospif(-2.0f * (float)i / (float)Mp, &sn, &cs);
    tw[i] = make_float2(cs, sn);
  }
  for (int i = tid; i < (L + 1) * kVolMaxHD; i += kAlignThreads) {
    const int l = i / kVolMaxHD, d = i % kVolMaxHD;
    Vs[i] = (d < HD) ? (float)p.V[l * HD + d] : 0.f;
  }
  __syncthreads();

  // Steps 1 and 1b: Y_d(m1, m2) = sum_l V_{l d} sum_h conj(a_{h,l}^{m1}) b_{h,l}^{m2}
  float2 Y[EPT][kVolMaxHD];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
#pragma unroll
    for (int d = 0; d < kVolMaxHD; ++d) Y[q][d] = make_float2(0.f, 0.f);
    const int e = tid + q * kAlignThreads;
    if (e < M * M) {
      const int i1 = e / M, i2 = e % M;
      const int l0 = max(abs(i1 - L), abs(i2 - L));
      for (int l = l0; l <= L; ++l) {
        float2 x = make_float2(0.f, 0.f);
        for (int h = 0; h < HC; ++h) {
          const float2 a = sa[(h * (L + 1) + l) * M + i1], b = sb[(h * (L + 1) + l) * M + i2];
          x.x = fmaf(a.x, b.x, fmaf(a.y, b.y, x.x));
          x.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, x.y));
        }
#pragma unroll
        for (int d = 0; d < kVolMaxHD; ++d) {
          const float v = Vs[l * kVolMaxHD + d];
          Y[q][d].x = fmaf(v, x.x, Y[q][d].x);
          Y[q][d].y = fmaf(v, x.y, Y[q][d].y);
        }
      }
    }
  }

  float run_best = -INFINITY;
  int run_arg = 0;
  const int lg = p.log2Mp;
  for (int bi = 0; bi < p.n_beta; ++bi) {
    // Step 2 into the zero-padded grid, rows and columns bit-reversed for the transform
    for (int i = tid; i < Mp * XP; i += kAlignThreads) buf[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const float* Tb = p.T + (size_t)bi * HD * M * M;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * kAlignThreads;
      if (e < M * M) {
        float2 xh = make_float2(0.f, 0.f);
#pragma unroll
        for (int d = 0; d < kVolMaxHD; ++d) {
          if (d < HD) {
            const float t = Tb[(size_t)d * M * M + e];
            xh.x = fmaf(t, Y[q][d].x, xh.x);
            xh.y = fmaf(t, Y[q][d].y, xh.y);
          }
        }
        const int m1 = (e / M - L + Mp) % Mp, m2 = (e % M - L + Mp) % Mp;
        const int r1 = (int)(__brev((unsigned)m1) >> (32 - lg)), r2 = (int)(__brev((unsigned)m2) >> (32 - lg));
        buf[r1 * XP + r2] = xh;
      }
    }
    __syncthreads();
    // Step 3: forward DFT along the m2 index (rows), then along m1 (columns)
    for (int dim = 0; dim < 2; ++dim) {
      for (int half = 1; half < Mp; half *= 2) {
        const int stride = Mp / (2 * half);
        for (int bf = tid; bf < Mp * Mp / 2; bf += kAlignThreads) {
          const int line = bf / (Mp / 2), k = bf % (Mp / 2);
          const int pos = k % half, grp = k / half;
          const int i0 = grp * 2 * half + pos, i1 = i0 + half;
          const int a0 = dim == 0 ? line * XP + i0 : i0 * XP + line;
          const int a1 = dim == 0 ? line * XP + i1 : i1 * XP + line;
          const float2 w = tw[pos * stride];
          const float2 u = buf[a0];
          const float2 v = cmul(buf[a1], w);
          buf[a0] = make_float2(u.x + v.x, u.y + v.y);
          buf[a1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
      }
    }
    // max / argmax over (alpha_a, gamma_c) of this beta, smallest index first
    float bv = -INFINITY;
    int ba = 0x7fffffff;
    for (int i = tid; i < Mp * Mp; i += kAlignThreads) {
      const int a = i / Mp, c = i % Mp;
      const float v = buf[a * XP + c].x;
      if (v > bv) {  // i increases per thread: ties keep the first
        bv = v;
        ba = i;
      }
    }
    argmax_warp_reduce(bv, ba, 32);
    if ((tid & 31) == 0) {
      rv[tid >> 5] = bv;
      ri[tid >> 5] = ba;
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
      if (bi == 0 || tb > run_best) {  // increasing beta: ties keep the earlier
        run_best = tb;
        run_arg = bi * Mp * Mp + ti;
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    p.best[(size_t)n * p.N_B + j] = run_best;
    p.arg[(size_t)n * p.N_B + j] = run_arg;
  }
}

size_t vol_align_smem(int HC, int L, int Mp) {
  const size_t LM = (size_t)(L + 1) * (2 * L + 1);
  return (2 * HC * LM + (size_t)Mp * (Mp + 1) + Mp / 2) * sizeof(float2) + 64 * sizeof(float) +
         (size_t)(L + 1) * kVolMaxHD * sizeof(float);
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
  vol_compress_kernel<<<(unsigned)((total + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(cp);
  return launch_status();
}

extern "C" int rsvd_align_volumes(const void* cA, int N_A, const void* cB, int N_B, int HC, int L, const double* V,
                                  int HD, const float* tables, int n_beta, int Mp, float* best, int32_t* arg,
                                  void* stream) {
  using namespace rsvd;
  if (!cA || !cB || !V || !tables || !best || !arg || N_A <= 0 || N_B <= 0 || HC <= 0 || L < 1 || HD <= 0 ||
      n_beta <= 0)
    return RSVD_EINVAL;
  if (L > kVolMaxL || HD > kVolMaxHD || HC > kVolMaxHC || HD > L + 1) return RSVD_EUNSUPPORTED;
  if (!(Mp == 16 || Mp == 32 || Mp == 64) || Mp < 2 * L + 1) return RSVD_EUNSUPPORTED;
  if ((long long)N_A * N_B > 0x7fffffffLL) return RSVD_EUNSUPPORTED;
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
  ap.Mp = Mp;
  int lg = 0;
  while ((1 << lg) < Mp) ++lg;
  ap.log2Mp = lg;
  const int M = 2 * L + 1;
  const int ept = (M * M + kAlignThreads - 1) / kAlignThreads;
  const size_t smem = vol_align_smem(HC, L, Mp);
  if (smem > 227 * 1024) return RSVD_EUNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto go = [&](auto kern) -> int {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return RSVD_ECUDA;
    kern<<<(unsigned)((long long)N_A * N_B), kAlignThreads, smem, st>>>(ap);
    return launch_status();
  };
  if (ept <= 2) return go(vol_align_kernel<2>);
  if (ept <= 3) return go(vol_align_kernel<3>);
  if (ept <= 5) return go(vol_align_kernel<5>);
  return RSVD_EUNSUPPORTED;  // (2L+1)^2 > 5 x 512: L > 24
}
