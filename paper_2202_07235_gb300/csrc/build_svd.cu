// rsvd_build_radial_svd: ring-ring kernel C (FP64) and its principal vectors.
//
// Paper section 3.3, eq. (Image_simple_kern) and section 3.4,
// eq. (image_cost_and_kern):  C_{rr'} = (1/N_B) sum_j sum_{q != 0}
// Re conj(beta_j(r,q)) beta_j(r',q), beta_j(r,q) = sqrt(w_r) b_j(k_r,q).
//
// The q-sum is evaluated without an FFT through Parseval's identity on each
// ring, sum_{q} conj(b(r,q)) b(r',q) = (1/Q) sum_psi conj(B(r,psi)) B(r',psi), minus the
// q = 0 term b(r,0) = (1/Q) sum_psi B(r,psi) (the ring mean). For the transform of a
// real image the psi and psi+pi samples are conjugate, so with M = Q/2:
//   G_{rr'}   = sum_j sum_{psi<M} Re conj(B_j(r,psi)) B_j(r',psi)
//   m_j(r)    = (2/Q) sum_{psi<M} Re B_j(r,psi)
//   C_{rr'}   = sqrt(w_r w_r') / N_B * [ (2/Q) G_{rr'} - sum_j m_j(r) m_j(r') ].
// kernel_partial: CTA (slice, tile) accumulates a 64x64 tile of C over a slice
// of templates (FP64, 4x4 register block per thread) into the workspace;
// kernel_reduce: sums the slices. jacobi_eig: cyclic Jacobi with the
// round-robin (tournament) ordering on one CTA, FP64, then sorting,
// sign-fixing and writing U and the eigenvalues.
#include <math.h>

#include <mutex>

#include "rsvd_internal.cuh"

namespace rsvd {
RSVD_HIDDEN int launch_jacobi(const double* C, double* A, double* V, int R, int H, double* U, double* eig, int batch,
                              cudaStream_t st);
namespace {

constexpr int kTile = 64;       // C tile edge
constexpr int kPsiChunk = 32;   // angles staged per step
constexpr int kThreads = 256;   // 16 x 16 threads, 4 x 4 entries each
constexpr int kMaxSlices = 304;
constexpr int kJacobiThreads = 1024;
constexpr int kMaxSweeps = 40;

struct BuildPlan {
  int tiles1d, ntiles, nslices;
  size_t off_partial, off_C, off_A, off_V, total;
};

BuildPlan make_plan(int R, int N_B) {
  BuildPlan pl{};
  pl.tiles1d = (R + kTile - 1) / kTile;
  pl.ntiles = pl.tiles1d * pl.tiles1d;
  int ns = kMaxSlices / pl.ntiles;
  if (ns < 1) ns = 1;
  if (ns > N_B) ns = N_B;
  pl.nslices = ns;
  const size_t rr = (size_t)R * R * sizeof(double);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  pl.off_partial = 0;
  pl.off_C = up((size_t)ns * rr);
  pl.off_A = pl.off_C + up(rr);
  pl.off_V = pl.off_A + up(rr);
  pl.total = pl.off_V + up(rr);
  return pl;
}

// kSplit: the two sums are kept apart (partial = sum_j (2/Q) G_j, partial + nslices R^2 =
// sum_j m_j m_j^T) for the translation-aware kernel, which weighs them differently.
template <bool kSplit>
__global__ void __launch_bounds__(kThreads) kernel_partial(const float2* __restrict__ B, int N_B, int R, int Q,
                                                           int tiles1d, int nslices, double* __restrict__ partial) {
  __shared__ float2 sr[kTile][kPsiChunk + 1];
  __shared__ float2 sc[kTile][kPsiChunk + 1];
  const int slice = blockIdx.x, tile = blockIdx.y;
  const int tr = tile / tiles1d, tc = tile % tiles1d;
  const int r0 = tr * kTile, c0 = tc * kTile;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int M = Q / 2;
  const int j_begin = (int)((long long)N_B * slice / nslices);
  const int j_end = (int)((long long)N_B * (slice + 1) / nslices);
  const double scale_g = 2.0 / (double)Q;
  double acc[4][4], acc2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = acc2[a][b] = 0.0;

  for (int j = j_begin; j < j_end; ++j) {
    const float2* Bj = B + (size_t)j * R * Q;
    double g[4][4];
    double mr[4] = {0, 0, 0, 0}, mc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) g[a][b] = 0.0;
    for (int p0 = 0; p0 < M; p0 += kPsiChunk) {
      __syncthreads();
      for (int i = threadIdx.x; i < kTile * kPsiChunk; i += kThreads) {
        const int rr = i / kPsiChunk, pp = i % kPsiChunk;
        const int psi = p0 + pp;
        const bool okp = psi < M;
        sr[rr][pp] = (okp && r0 + rr < R) ? Bj[(size_t)(r0 + rr) * Q + psi] : make_float2(0.f, 0.f);
        sc[rr][pp] = (okp && c0 + rr < R) ? Bj[(size_t)(c0 + rr) * Q + psi] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll 4
      for (int pp = 0; pp < kPsiChunk; ++pp) {
        double xr[4], xi[4], yr[4], yi[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float2 u = sr[ty * 4 + a][pp];
          const float2 v = sc[tx * 4 + a][pp];
          xr[a] = u.x;
          xi[a] = u.y;
          yr[a] = v.x;
          yi[a] = v.y;
          mr[a] += xr[a];
          mc[a] += yr[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) g[a][b] = fma(xr[a], yr[b], fma(xi[a], yi[b], g[a][b]));
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (kSplit) {
          acc[a][b] += scale_g * g[a][b];
          acc2[a][b] += (scale_g * mr[a]) * (scale_g * mc[b]);
        } else {
          acc[a][b] += scale_g * g[a][b] - (scale_g * mr[a]) * (scale_g * mc[b]);
        }
      }
  }
  double* out = partial + (size_t)slice * R * R;
  double* out2 = partial + ((size_t)nslices + slice) * R * R;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = r0 + ty * 4 + a;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (r < R && c < R) {
        out[(size_t)r * R + c] = acc[a][b];
        if (kSplit) out2[(size_t)r * R + c] = acc2[a][b];
      }
    }
  }
}

struct ReduceParams {
  const double* partial;
  double* C;
  int R, nslices, N_B;
  double sw[kMaxR];
};

__global__ void kernel_reduce(const __grid_constant__ ReduceParams p) {
  const int RR = p.R * p.R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RR; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < p.nslices; ++k) s += p.partial[(size_t)k * RR + i];
    const int r = i / p.R, c = i % p.R;
    p.C[i] = s * p.sw[r] * p.sw[c] / (double)p.N_B;
  }
}

// Position of element i in round k of the round-robin schedule over n (even)
// indices: index 0 stays, the others rotate.
__device__ __forceinline__ int rr_member(int pos, int k, int n) { return pos == 0 ? 0 : ((pos - 1 + k) % (n - 1)) + 1; }

__global__ void __launch_bounds__(kJacobiThreads) jacobi_eig(const double* __restrict__ C, double* A, double* V, int R,
                                                              int H, double* __restrict__ U, double* __restrict__ eig,
                                                              int use_smem, int* status) {
  extern __shared__ __align__(16) double jsm[];
  __shared__ double cs_c[kMaxR / 2 + 1], cs_s[kMaxR / 2 + 1];
  // batched use (one CTA per matrix): matrix blockIdx.x of consecutive R x R blocks
  {
    const size_t b = blockIdx.x;
    C += b * R * R;
    A += b * R * R;
    V += b * R * R;
    U += b * R * H;
    eig += b * R;
  }
  __shared__ int pr_p[kMaxR / 2 + 1], pr_q[kMaxR / 2 + 1];
  __shared__ int rotated;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int n = (R % 2) ? R + 1 : R;  // padded to even; index R (if any) is a dummy
  if (use_smem) {
    A = jsm;
    V = jsm + (size_t)R * R;
  }
  for (int i = tid; i < R * R; i += nth) {
    const int r = i / R, c = i % R;
    A[i] = 0.5 * (C[i] + C[(size_t)c * R + r]);  // exact symmetry
    V[i] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int npairs = n / 2;
  __shared__ double anorm;
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < R; ++i) m = fmax(m, fabs(A[(size_t)i * R + i]));
    anorm = m;
  }
  __syncthreads();
  // rotate while |a_pq| exceeds both a relative (to sqrt(a_pp a_qq)) and an
  // absolute (to the largest diagonal entry) rounding-level threshold
  // below a few ulp of the largest diagonal the off-diagonals are rounding noise of
  // the rotations themselves (kernels with near-zero rings, e.g. at CTF zeros)
  const double abs_floor = 1e-15 * anorm;
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {
      // rotation parameters (Golub & Van Loan, symmetric Schur 2x2)
      for (int i = tid; i < npairs; i += nth) {
        int pp = rr_member(i, k, n), qq = rr_member(n - 1 - i, k, n);
        if (pp > qq) {
          const int tmp = pp;
          pp = qq;
          qq = tmp;
        }
        double c = 1.0, s = 0.0;
        if (qq < R) {
          const double apq = A[(size_t)pp * R + qq];
          const double app = A[(size_t)pp * R + pp], aqq = A[(size_t)qq * R + qq];
          if (fabs(apq) > fmax(1e-15 * sqrt(fabs(app * aqq)), abs_floor) && apq != 0.0) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
            rotated = 1;
          }
        }
        cs_c[i] = c;
        cs_s[i] = s;
        pr_p[i] = pp;
        pr_q[i] = qq;
      }
      __syncthreads();
      // columns of A and V: A <- A J, V <- V J
      for (int idx = tid; idx < npairs * R; idx += nth) {
        const int i = idx / R, r = idx % R;
        const int pp = pr_p[i], qq = pr_q[i];
        if (qq >= R || cs_s[i] == 0.0) continue;
        const double c = cs_c[i], s = cs_s[i];
        const double ap = A[(size_t)r * R + pp], aq = A[(size_t)r * R + qq];
        A[(size_t)r * R + pp] = c * ap - s * aq;
        A[(size_t)r * R + qq] = s * ap + c * aq;
        const double vp = V[(size_t)r * R + pp], vq = V[(size_t)r * R + qq];
        V[(size_t)r * R + pp] = c * vp - s * vq;
        V[(size_t)r * R + qq] = s * vp + c * vq;
      }
      __syncthreads();
      // rows of A: A <- J^T A
      for (int idx = tid; idx < npairs * R; idx += nth) {
        const int i = idx / R, cidx = idx % R;
        const int pp = pr_p[i], qq = pr_q[i];
        if (qq >= R || cs_s[i] == 0.0) continue;
        const double c = cs_c[i], s = cs_s[i];
        const double ap = A[(size_t)pp * R + cidx], aq = A[(size_t)qq * R + cidx];
        A[(size_t)pp * R + cidx] = c * ap - s * aq;
        A[(size_t)qq * R + cidx] = s * ap + c * aq;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  if (sweep >= kMaxSweeps && tid == 0) record(status, kDevNoConverge);
  // sort by decreasing eigenvalue (stable on index), fix signs, write out
  for (int i = tid; i < R; i += nth) {
    const double li = A[(size_t)i * R + i];
    int rank = 0;
    for (int j = 0; j < R; ++j) {
      const double lj = A[(size_t)j * R + j];
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    eig[rank] = li;
    if (rank < H) {
      int imax = 0;
      double vmax = -1.0;
      for (int r = 0; r < R; ++r) {
        const double v = fabs(V[(size_t)r * R + i]);
        if (v > vmax) {
          vmax = v;
          imax = r;
        }
      }
      const double sg = V[(size_t)imax * R + i] < 0.0 ? -1.0 : 1.0;
      for (int r = 0; r < R; ++r) U[(size_t)r * H + rank] = sg * V[(size_t)r * R + i];
    }
  }
}

// ---------------------------------------------------------------------------
// Eigen-decomposition for R <= 64 with most of the work in FP32 (the part's
// FP64 rate is 1/64 of its FP32 rate), finished in FP64: an FP32 cyclic Jacobi
// gives an approximate eigenbasis V0; one FP64 Newton-Schulz step
// V0 <- V0 (3 I - V0^T V0) / 2 makes it orthonormal to rounding; the FP64
// Jacobi of the nearly diagonal A1 = V0^T C V0 (a couple of sweeps) gives V1,
// and U = V0 V1 with the eigenvalues on the diagonal. Everything stays in
// shared memory (four R x R FP64 buffers); one CTA per matrix.
// ---------------------------------------------------------------------------
constexpr int kMixedMaxR = 64;

// Z = op(X) Y for R x R row-major matrices in shared memory (op = transpose if tx)
__device__ __forceinline__ void smem_mm(const double* X, bool tx, const double* Y, double* Z, int R) {
  for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
    const int i = idx / R, j = idx % R;
    double acc = 0.0;
    if (tx) {
      for (int k = 0; k < R; ++k) acc = fma(X[k * R + i], Y[k * R + j], acc);
    } else {
      for (int k = 0; k < R; ++k) acc = fma(X[i * R + k], Y[k * R + j], acc);
    }
    Z[idx] = acc;
  }
}

// Cyclic Jacobi sweeps in precision F on symmetric A (R x R) accumulating V;
// returns the number of sweeps run (max_sweeps if still rotating).
template <typename F>
__device__ int sym_jacobi(F* A, F* V, int R, int max_sweeps, F rel, F absfloor, F* cs_c, F* cs_s, int* pr_p,
                          int* pr_q, int* rotated) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int n = (R % 2) ? R + 1 : R, npairs = n / 2;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {
      for (int i = tid; i < npairs; i += nth) {
        int pp = rr_member(i, k, n), qq = rr_member(n - 1 - i, k, n);
        if (pp > qq) {
          const int tmp = pp;
          pp = qq;
          qq = tmp;
        }
        F c = 1, s = 0;
        if (qq < R) {
          const F apq = A[pp * R + qq], app = A[pp * R + pp], aqq = A[qq * R + qq];
          if (fabs(apq) > fmax(rel * sqrt(fabs(app * aqq)), absfloor) && apq != F(0)) {
            const F tau = (aqq - app) / (F(2) * apq);
            const F t = (tau >= F(0) ? F(1) : F(-1)) / (fabs(tau) + sqrt(F(1) + tau * tau));
            c = F(1) / sqrt(F(1) + t * t);
            s = t * c;
            *rotated = 1;
          }
        }
        cs_c[i] = c;
        cs_s[i] = s;
        pr_p[i] = pp;
        pr_q[i] = qq;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * R; idx += nth) {  // A <- A J, V <- V J
        const int i = idx / R, r = idx % R;
        const int pp = pr_p[i], qq = pr_q[i];
        if (qq >= R || cs_s[i] == F(0)) continue;
        const F c = cs_c[i], s = cs_s[i];
        const F ap = A[r * R + pp], aq = A[r * R + qq];
        A[r * R + pp] = c * ap - s * aq;
        A[r * R + qq] = s * ap + c * aq;
        const F vp = V[r * R + pp], vq = V[r * R + qq];
        V[r * R + pp] = c * vp - s * vq;
        V[r * R + qq] = s * vp + c * vq;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * R; idx += nth) {  // A <- J^T A
        const int i = idx / R, col = idx % R;
        const int pp = pr_p[i], qq = pr_q[i];
        if (qq >= R || cs_s[i] == F(0)) continue;
        const F c = cs_c[i], s = cs_s[i];
        const F ap = A[pp * R + col], aq = A[qq * R + col];
        A[pp * R + col] = c * ap - s * aq;
        A[qq * R + col] = s * ap + c * aq;
      }
      __syncthreads();
    }
    if (!*rotated) break;
    __syncthreads();
  }
  return sweep;
}

__global__ void __launch_bounds__(kJacobiThreads) jacobi_mixed(const double* __restrict__ C, int R, int H,
                                                                double* __restrict__ U, double* __restrict__ eig,
                                                                int* status) {
  extern __shared__ __align__(16) double jm[];
  __shared__ double cd_c[kMixedMaxR / 2 + 1], cd_s[kMixedMaxR / 2 + 1];
  __shared__ float cf_c[kMixedMaxR / 2 + 1], cf_s[kMixedMaxR / 2 + 1];
  __shared__ int pr_p[kMixedMaxR / 2 + 1], pr_q[kMixedMaxR / 2 + 1];
  __shared__ int rotated;
  __shared__ double anorm;
  {
    const size_t b = blockIdx.x;  // batched: one matrix per CTA
    C += b * R * R;
    U += b * R * H;
    eig += b * R;
  }
  const int tid = threadIdx.x, nth = blockDim.x, RR = R * R;
  double* D0 = jm;
  double* D1 = jm + RR;
  double* D2 = jm + 2 * RR;
  double* D3 = jm + 3 * RR;
  float* Af = reinterpret_cast<float*>(D0);  // FP32 stage: A and V in D0's space
  float* Vf = Af + RR;
  for (int i = tid; i < RR; i += nth) {
    const int r = i / R, c = i % R;
    Af[i] = (float)(0.5 * (C[i] + C[(size_t)c * R + r]));
    Vf[i] = (r == c) ? 1.f : 0.f;
  }
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < R; ++i) m = fmax(m, fabs(C[(size_t)i * R + i]));
    anorm = m;
  }
  __syncthreads();
  // FP32 stage: off-diagonals down to about single-precision rounding of the largest
  // diagonal entry (the FP64 stage finishes; below that FP32 sweeps only stir noise)
  (void)sym_jacobi<float>(Af, Vf, R, 12, 1e-5f, 1e-6f * (float)anorm, cf_c, cf_s, pr_p, pr_q, &rotated);
  __syncthreads();
  for (int i = tid; i < RR; i += nth) D1[i] = (double)Vf[i];
  __syncthreads();
  // one Newton-Schulz step: V0 = D1 (3 I - D1^T D1) / 2 -> D3
  smem_mm(D1, true, D1, D2, R);
  __syncthreads();
  for (int i = tid; i < RR; i += nth) {
    const int r = i / R, c = i % R;
    D2[i] = (r == c ? 1.5 : 0.0) - 0.5 * D2[i];
  }
  __syncthreads();
  smem_mm(D1, false, D2, D3, R);
  __syncthreads();
  // A1 = V0^T C V0 (C symmetrised into D0), symmetrised into D1
  for (int i = tid; i < RR; i += nth) {
    const int r = i / R, c = i % R;
    D0[i] = 0.5 * (C[i] + C[(size_t)c * R + r]);
  }
  __syncthreads();
  smem_mm(D0, false, D3, D1, R);
  __syncthreads();
  smem_mm(D3, true, D1, D2, R);
  __syncthreads();
  for (int i = tid; i < RR; i += nth) {
    const int r = i / R, c = i % R;
    D1[i] = 0.5 * (D2[i] + D2[c * R + r]);
    D0[i] = (r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  // FP64 stage on the nearly diagonal A1 (D1) with V1 (D0). Off-diagonals below
  // 1e-13 of the largest diagonal entry are left: they move an eigenvalue by at
  // most R x that (about 1e-11 of the largest) and a vector with spectral gap g
  // by about that / g, while sweeping them to rounding level costs most of the
  // time for kernels whose many small eigenvalues sit below FP32 resolution.
  const int sweeps = sym_jacobi<double>(D1, D0, R, kMaxSweeps, 1e-15, 1e-13 * anorm, cd_c, cd_s, pr_p, pr_q,
                                        &rotated);
  if (sweeps >= kMaxSweeps && tid == 0) record(status, kDevNoConverge);
  __syncthreads();
  smem_mm(D3, false, D0, D2, R);  // eigenvectors V0 V1
  __syncthreads();
  // sort by decreasing eigenvalue (stable on index), fix signs, write out
  for (int i = tid; i < R; i += nth) {
    const double li = D1[i * R + i];
    int rank = 0;
    for (int j = 0; j < R; ++j) {
      const double lj = D1[j * R + j];
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    eig[rank] = li;
    if (rank < H) {
      int imax = 0;
      double vmax = -1.0;
      for (int r = 0; r < R; ++r) {
        const double v = fabs(D2[r * R + i]);
        if (v > vmax) {
          vmax = v;
          imax = r;
        }
      }
      const double sg = D2[imax * R + i] < 0.0 ? -1.0 : 1.0;
      for (int r = 0; r < R; ++r) U[(size_t)r * H + rank] = sg * D2[r * R + i];
    }
  }
}

}  // namespace
}  // namespace rsvd

extern "C" size_t rsvd_build_workspace_bytes(int R, int Q, int N_B) {
  if (R <= 0 || R > rsvd::kMaxR || Q <= 0 || N_B <= 0) return 0;
  return rsvd::make_plan(R, N_B).total;
}

extern "C" int rsvd_build_radial_svd(int R, int Q, const double* w, const void* templates, int N_B, int H, double* U,
                                     double* eig, void* workspace, size_t workspace_bytes, void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!w || !templates || !U || !eig || N_B <= 0) return RSVD_EINVAL;
  if (((uintptr_t)templates & 7u) || ((uintptr_t)U & 7u) || ((uintptr_t)eig & 7u)) return RSVD_EINVAL;
  const BuildPlan pl = make_plan(R, N_B);
  if (!workspace || workspace_bytes < pl.total || ((uintptr_t)workspace & 255u)) return RSVD_EWORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws + pl.off_partial);
  double* C = reinterpret_cast<double*>(ws + pl.off_C);
  double* A = reinterpret_cast<double*>(ws + pl.off_A);
  double* V = reinterpret_cast<double*>(ws + pl.off_V);

  dim3 grid(pl.nslices, pl.ntiles);
  kernel_partial<false><<<grid, kThreads, 0, st>>>(static_cast<const float2*>(templates), N_B, R, Q, pl.tiles1d,
                                                   pl.nslices, partial);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  ReduceParams rp{};
  rp.partial = partial;
  rp.C = C;
  rp.R = R;
  rp.nslices = pl.nslices;
  rp.N_B = N_B;
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    rp.sw[r] = sqrt(w[r]);
  }
  kernel_reduce<<<(R * R + 255) / 256, 256, 0, st>>>(rp);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  return launch_jacobi(C, A, V, R, H, U, eig, 1, st);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of rsvd_build_radial_svd.
//
// Some callers cannot allocate device memory: a host application that hands
// this library raw pointers from inside a plugin or callback has no allocator
// of its own to call, and a service that fixes its device footprint at start-up
// must not grow it (or fragment a caching allocator) when the principal
// vectors are rebuilt. For them the scratch of the build (per-slice partial
// sums of C, C itself and the two Jacobi matrices) lives in a fixed
// file-scope device array that every GPU loading the library holds until the
// process exits. The array keeps the last call's contents; every word a call
// reads is first written by that same call, so nothing needs clearing. All
// calls share it: calls that overlap on the GPU (different streams, or
// different host threads on one device) race and must be serialised by the
// caller.
// ---------------------------------------------------------------------------
namespace rsvd {
namespace {

// 1 MiB: enough for the four R x R FP64 matrices of the build up to R = 181
// (fewer template slices are used than in the workspace entry point).
constexpr size_t kStaticScratchBytes = (size_t)1 << 20;
static __device__ __align__(256) unsigned char g_build_scratch[kStaticScratchBytes];

BuildPlan make_plan_capped(int R, int N_B, size_t cap) {
  BuildPlan pl{};
  pl.tiles1d = (R + kTile - 1) / kTile;
  pl.ntiles = pl.tiles1d * pl.tiles1d;
  const size_t rr = (size_t)R * R * sizeof(double);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  int ns = kMaxSlices / pl.ntiles;
  if (ns < 1) ns = 1;
  if (ns > N_B) ns = N_B;
  const size_t fixed = 3 * up(rr);
  while (ns > 1 && up((size_t)ns * rr) + fixed > cap) --ns;
  pl.nslices = ns;
  pl.off_partial = 0;
  pl.off_C = up((size_t)ns * rr);
  pl.off_A = pl.off_C + up(rr);
  pl.off_V = pl.off_A + up(rr);
  pl.total = pl.off_V + up(rr);
  return pl;
}

// Device address of g_build_scratch on the current device, looked up once per
// device (the host-side name of a __device__ array is only a stand-in).
int static_scratch(void** out) {
  static std::mutex mu;
  static void* ptrs[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RSVD_ECUDA;
  if (dev < 0 || dev >= 64) return RSVD_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_build_scratch) != cudaSuccess || p == nullptr) return RSVD_ECUDA;
    ptrs[dev] = p;
  }
  *out = ptrs[dev];
  return RSVD_OK;
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_build_radial_svd_noalloc(int R, int Q, const double* w, const void* templates, int N_B, int H,
                                             double* U, double* eig, void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!w || !templates || !U || !eig || N_B <= 0) return RSVD_EINVAL;
  if (((uintptr_t)templates & 7u) || ((uintptr_t)U & 7u) || ((uintptr_t)eig & 7u)) return RSVD_EINVAL;
  const BuildPlan pl = make_plan_capped(R, N_B, kStaticScratchBytes);
  if (pl.total > kStaticScratchBytes) return RSVD_EUNSUPPORTED;  // R too large for the fixed scratch
  ReduceParams rp{};
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    rp.sw[r] = sqrt(w[r]);
  }
  void* scratch = nullptr;
  if ((rc = static_scratch(&scratch)) != RSVD_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(scratch);
  double* partial = reinterpret_cast<double*>(ws + pl.off_partial);
  double* C = reinterpret_cast<double*>(ws + pl.off_C);
  double* A = reinterpret_cast<double*>(ws + pl.off_A);
  double* V = reinterpret_cast<double*>(ws + pl.off_V);

  dim3 grid(pl.nslices, pl.ntiles);
  kernel_partial<false><<<grid, kThreads, 0, st>>>(static_cast<const float2*>(templates), N_B, R, Q, pl.tiles1d,
                                                   pl.nslices, partial);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  rp.partial = partial;
  rp.C = C;
  rp.R = R;
  rp.nslices = pl.nslices;
  rp.N_B = N_B;
  kernel_reduce<<<(R * R + 255) / 256, 256, 0, st>>>(rp);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  const size_t need = (size_t)2 * R * R * sizeof(double);
  const int use_smem = need <= 160 * 1024 ? 1 : 0;
  const size_t smem = use_smem ? need : 0;
  if (use_smem &&
      cudaFuncSetAttribute(jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RSVD_ECUDA;
  jacobi_eig<<<1, kJacobiThreads, smem, st>>>(C, A, V, R, H, U, eig, use_smem, status_word());
  return launch_status();
}

// ---------------------------------------------------------------------------
// Translation-aware kernel (section 5, eq. Image_single_cost_with_translations):
// the objective averaged over the Q grid rotations and a distribution of
// translations {delta_t, p_t} of the target is quadratic in u with kernel
//   C_{rr'} = sqrt(w_r w_r') / N_B * sum_j [ S_j(r,r') Phi_{rr'} - m_j(r) m_j(r') Psi_{rr'} ],
//   S_j(r,r')  = sum_q conj(b_j(r,q)) b_j(r',q)   (all q; Parseval on each ring),
//   m_j(r)     = b_j(r,0)                         (ring mean),
//   Phi_{rr'}  = (1/Q) sum_psi sum_t p_t cos((k_r - k_r') delta_t.n(psi)),
//   Psi_{rr'}  = (1/Q) sum_psi Re conj(phi_r(psi)) phi_r'(psi),  phi_r(psi) = sum_t p_t exp(-i k_r delta_t.n(psi)),
// (real parts: S_j and m_j are real for the transform of a real image). With the
// single translation delta = 0 it is the kernel of rsvd_build_radial_svd.
// ---------------------------------------------------------------------------
namespace rsvd {
namespace {

constexpr int kMomTile = 16;
constexpr int kMomChunk = 32;

struct MomentParams {
  double k[kMaxR];
  double dx[kMaxT], dy[kMaxT], pt[kMaxT];
  int R, Q, T;
};

// phi[r][q] = sum_t p_t exp(-i k_r rho_t(q)), rho_t(q) = dx_t cos psi_q + dy_t sin psi_q.
__global__ void kernel_phi(const __grid_constant__ MomentParams p, double2* __restrict__ phi) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.R * p.Q) return;
  const int r = i / p.Q, q = i % p.Q;
  double sp, cp;
  sincospi(2.0 * q / p.Q, &sp, &cp);
  double re = 0.0, im = 0.0;
  for (int t = 0; t < p.T; ++t) {
    double s, c;
    sincos(p.k[r] * (p.dx[t] * cp + p.dy[t] * sp), &s, &c);
    re += p.pt[t] * c;
    im -= p.pt[t] * s;
  }
  phi[i] = make_double2(re, im);
}

// Phi and Psi on 16 x 16 tiles of (r, r'); exp(-i k rho) of the tile's rows and
// columns is staged per (translation, chunk of angles) in shared memory.
__global__ void __launch_bounds__(kMomTile * kMomTile) kernel_moments(const __grid_constant__ MomentParams p,
                                                                     const double2* __restrict__ phi,
                                                                     double* __restrict__ Phi,
                                                                     double* __restrict__ Psi) {
  __shared__ double2 er[kMomTile][kMomChunk + 1], ec[kMomTile][kMomChunk + 1];
  __shared__ double cps[kMomChunk], sps[kMomChunk];
  const int tiles1d = (p.R + kMomTile - 1) / kMomTile;
  const int r0 = (blockIdx.x / tiles1d) * kMomTile, c0 = (blockIdx.x % tiles1d) * kMomTile;
  const int ty = threadIdx.x / kMomTile, tx = threadIdx.x % kMomTile;
  const int r = r0 + ty, c = c0 + tx;
  double acc = 0.0;
  for (int t = 0; t < p.T; ++t) {
    for (int q0 = 0; q0 < p.Q; q0 += kMomChunk) {
      __syncthreads();
      if (threadIdx.x < kMomChunk) {
        double sp = 0.0, cp = 0.0;
        if (q0 + threadIdx.x < p.Q) sincospi(2.0 * (q0 + threadIdx.x) / p.Q, &sp, &cp);
        cps[threadIdx.x] = cp;
        sps[threadIdx.x] = sp;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < 2 * kMomTile * kMomChunk; i += blockDim.x) {
        const int side = i / (kMomTile * kMomChunk), rem = i % (kMomTile * kMomChunk);
        const int row = rem / kMomChunk, qq = rem % kMomChunk;
        const int rr = (side == 0 ? r0 : c0) + row;
        double2 e = make_double2(0.0, 0.0);
        if (rr < p.R && q0 + qq < p.Q) {
          double s, cc;
          sincos(p.k[rr] * (p.dx[t] * cps[qq] + p.dy[t] * sps[qq]), &s, &cc);
          e = make_double2(cc, -s);
        }
        if (side == 0)
          er[row][qq] = e;
        else
          ec[row][qq] = e;
      }
      __syncthreads();
      double part = 0.0;
#pragma unroll 8
      for (int qq = 0; qq < kMomChunk; ++qq) part += er[ty][qq].x * ec[tx][qq].x + er[ty][qq].y * ec[tx][qq].y;
      acc += p.pt[t] * part;
    }
  }
  if (r < p.R && c < p.R) {
    double ps = 0.0;
    for (int q = 0; q < p.Q; ++q) {
      const double2 a = phi[(size_t)r * p.Q + q], b = phi[(size_t)c * p.Q + q];
      ps += a.x * b.x + a.y * b.y;
    }
    Phi[(size_t)r * p.R + c] = acc / p.Q;
    Psi[(size_t)r * p.R + c] = ps / p.Q;
  }
}

struct ReduceTParams {
  const double* partial;  // [2 nslices][R][R]
  const double* Phi;
  const double* Psi;
  double* C;
  int R, nslices, N_B;
  double sw[kMaxR];
};

__global__ void kernel_reduce_translated(const __grid_constant__ ReduceTParams p) {
  const int RR = p.R * p.R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < RR; i += gridDim.x * blockDim.x) {
    double g = 0.0, m = 0.0;
    for (int k = 0; k < p.nslices; ++k) {
      g += p.partial[(size_t)k * RR + i];
      m += p.partial[((size_t)p.nslices + k) * RR + i];
    }
    const int r = i / p.R, c = i % p.R;
    p.C[i] = (g * p.Phi[i] - m * p.Psi[i]) * p.sw[r] * p.sw[c] / (double)p.N_B;
  }
}

struct BuildTPlan {
  BuildPlan base;
  size_t off_Phi, off_Psi, off_phi, total;
};

BuildTPlan make_plan_translated(int R, int Q, int N_B) {
  BuildTPlan t{};
  t.base = make_plan(R, N_B);
  const size_t rr = (size_t)R * R * sizeof(double);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  // the partial sums take two slices' worth per slice (the two sums kept apart)
  const size_t extra = up((size_t)t.base.nslices * rr);
  t.base.off_C += extra;
  t.base.off_A += extra;
  t.base.off_V += extra;
  t.base.total += extra;
  t.off_Phi = t.base.total;
  t.off_Psi = t.off_Phi + up(rr);
  t.off_phi = t.off_Psi + up(rr);
  t.total = t.off_phi + up((size_t)R * Q * sizeof(double2));
  return t;
}

}  // namespace
}  // namespace rsvd

extern "C" size_t rsvd_build_translated_workspace_bytes(int R, int Q, int N_B) {
  if (R <= 0 || R > rsvd::kMaxR || Q <= 0 || N_B <= 0) return 0;
  return rsvd::make_plan_translated(R, Q, N_B).total;
}

extern "C" int rsvd_build_radial_svd_translated(int R, int Q, const double* k, const double* w, const void* templates,
                                                int N_B, const double* deltas, const double* weights, int T, int H,
                                                double* U, double* eig, void* workspace, size_t workspace_bytes,
                                                void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!k || !w || !templates || !U || !eig || !deltas || N_B <= 0 || T <= 0) return RSVD_EINVAL;
  if (T > kMaxT) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)templates & 7u) || ((uintptr_t)U & 7u) || ((uintptr_t)eig & 7u)) return RSVD_EINVAL;
  const BuildTPlan pl = make_plan_translated(R, Q, N_B);
  if (!workspace || workspace_bytes < pl.total || ((uintptr_t)workspace & 255u)) return RSVD_EWORKSPACE;
  MomentParams mp{};
  mp.R = R;
  mp.Q = Q;
  mp.T = T;
  double psum = 0.0;
  for (int t = 0; t < T; ++t) {
    const double pw = weights ? weights[t] : 1.0;
    if (!(pw >= 0.0) || !isfinite(deltas[2 * t]) || !isfinite(deltas[2 * t + 1])) return RSVD_EINVAL;
    mp.dx[t] = deltas[2 * t];
    mp.dy[t] = deltas[2 * t + 1];
    mp.pt[t] = pw;
    psum += pw;
  }
  if (!(psum > 0.0)) return RSVD_EINVAL;
  for (int t = 0; t < T; ++t) mp.pt[t] /= psum;
  ReduceTParams rp{};
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    mp.k[r] = k[r];
    rp.sw[r] = sqrt(w[r]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws + pl.base.off_partial);
  double* C = reinterpret_cast<double*>(ws + pl.base.off_C);
  double* A = reinterpret_cast<double*>(ws + pl.base.off_A);
  double* V = reinterpret_cast<double*>(ws + pl.base.off_V);
  double* Phi = reinterpret_cast<double*>(ws + pl.off_Phi);
  double* Psi = reinterpret_cast<double*>(ws + pl.off_Psi);
  double2* phi = reinterpret_cast<double2*>(ws + pl.off_phi);

  dim3 grid(pl.base.nslices, pl.base.ntiles);
  kernel_partial<true><<<grid, kThreads, 0, st>>>(static_cast<const float2*>(templates), N_B, R, Q, pl.base.tiles1d,
                                                  pl.base.nslices, partial);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  kernel_phi<<<(R * Q + 255) / 256, 256, 0, st>>>(mp, phi);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  const int mt = (R + kMomTile - 1) / kMomTile;
  kernel_moments<<<mt * mt, kMomTile * kMomTile, 0, st>>>(mp, phi, Phi, Psi);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  rp.partial = partial;
  rp.Phi = Phi;
  rp.Psi = Psi;
  rp.C = C;
  rp.R = R;
  rp.nslices = pl.base.nslices;
  rp.N_B = N_B;
  kernel_reduce_translated<<<(R * R + 255) / 256, 256, 0, st>>>(rp);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  return launch_jacobi(C, A, V, R, H, U, eig, 1, st);
}

// ---------------------------------------------------------------------------
// One kernel per CTF (section 3.5: the targets of micrograph g are the
// templates corrected with its CTF, and the kernel of eq. image_cost_and_kern is
// built per group). An isotropic CTF multiplies ring r by ctf_g(k_r), so the
// group kernel is C_g = diag(ctf_g) C diag(ctf_g) with C the kernel of the
// uncorrected templates, and the CTF-corrected targets compress with
// diag(ctf_g) U_g. C is built once; the G eigen-decompositions run as one
// batched Jacobi launch (one CTA per group).
// ---------------------------------------------------------------------------
namespace rsvd {
namespace {

__global__ void kernel_scale_groups(const double* __restrict__ C, const double* __restrict__ ctf, int R, int G,
                                    double* __restrict__ Cg) {
  const long long RR = (long long)R * R;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < RR * G; i += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(i / RR);
    const int rc = (int)(i % RR);
    const int r = rc / R, c = rc % R;
    Cg[i] = ctf[(size_t)g * R + r] * ctf[(size_t)g * R + c] * C[rc];
  }
}

__global__ void kernel_scale_targets(const double* __restrict__ U, const double* __restrict__ ctf, int R, int H, int G,
                                     double* __restrict__ Ut) {
  const long long n = (long long)G * R * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long gr = i / H;  // g * R + r
    Ut[i] = ctf[gr] * U[i];
  }
}

struct BuildGPlan {
  BuildPlan base;
  size_t off_Cg, off_Ag, off_Vg, total;
};

BuildGPlan make_plan_grouped(int R, int N_B, int G) {
  BuildGPlan t{};
  t.base = make_plan(R, N_B);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t grr = (size_t)G * R * R * sizeof(double);
  t.off_Cg = t.base.total;
  t.off_Ag = t.off_Cg + up(grr);
  t.off_Vg = t.off_Ag + up(grr);
  t.total = t.off_Vg + up(grr);
  return t;
}

}  // namespace
}  // namespace rsvd

extern "C" size_t rsvd_build_grouped_workspace_bytes(int R, int Q, int N_B, int G) {
  if (R <= 0 || R > rsvd::kMaxR || Q <= 0 || N_B <= 0 || G <= 0) return 0;
  return rsvd::make_plan_grouped(R, N_B, G).total;
}

extern "C" int rsvd_build_radial_svd_grouped(int R, int Q, const double* w, const void* templates, int N_B,
                                             const double* ctf, int G, int H, double* U, double* U_targets,
                                             double* eig, void* workspace, size_t workspace_bytes, void* stream) {
  using namespace rsvd;
  int rc = check_grid(R, Q, H);
  if (rc != RSVD_OK) return rc;
  if (!w || !templates || !ctf || !U || !eig || N_B <= 0 || G <= 0) return RSVD_EINVAL;
  if (G > 65535) return RSVD_EUNSUPPORTED;
  if (((uintptr_t)templates & 7u) || ((uintptr_t)U & 7u) || ((uintptr_t)eig & 7u) || ((uintptr_t)ctf & 7u) ||
      ((uintptr_t)U_targets & 7u))
    return RSVD_EINVAL;
  const BuildGPlan pl = make_plan_grouped(R, N_B, G);
  if (!workspace || workspace_bytes < pl.total || ((uintptr_t)workspace & 255u)) return RSVD_EWORKSPACE;
  ReduceParams rp{};
  for (int r = 0; r < R; ++r) {
    if (!(w[r] >= 0.0)) return RSVD_EINVAL;
    rp.sw[r] = sqrt(w[r]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  double* partial = reinterpret_cast<double*>(ws + pl.base.off_partial);
  double* C = reinterpret_cast<double*>(ws + pl.base.off_C);
  double* Cg = reinterpret_cast<double*>(ws + pl.off_Cg);
  double* Ag = reinterpret_cast<double*>(ws + pl.off_Ag);
  double* Vg = reinterpret_cast<double*>(ws + pl.off_Vg);

  dim3 grid(pl.base.nslices, pl.base.ntiles);
  kernel_partial<false><<<grid, kThreads, 0, st>>>(static_cast<const float2*>(templates), N_B, R, Q, pl.base.tiles1d,
                                                   pl.base.nslices, partial);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  rp.partial = partial;
  rp.C = C;
  rp.R = R;
  rp.nslices = pl.base.nslices;
  rp.N_B = N_B;
  kernel_reduce<<<(R * R + 255) / 256, 256, 0, st>>>(rp);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  kernel_scale_groups<<<256, 256, 0, st>>>(C, ctf, R, G, Cg);
  if ((rc = launch_status()) != RSVD_OK) return rc;
  if ((rc = launch_jacobi(Cg, Ag, Vg, R, H, U, eig, G, st)) != RSVD_OK) return rc;
  if (U_targets) {
    kernel_scale_targets<<<256, 256, 0, st>>>(U, ctf, R, H, G, U_targets);
    if ((rc = launch_status()) != RSVD_OK) return rc;
  }
  return RSVD_OK;
}

namespace rsvd {

// Jacobi eigen-solver of `batch` consecutive R x R symmetric matrices (one CTA
// each): U [batch][R][H] leading vectors, eig [batch][R] decreasing.
RSVD_HIDDEN int launch_jacobi(const double* C, double* A, double* V, int R, int H, double* U, double* eig, int batch,
                              cudaStream_t st) {
  if (R <= kMixedMaxR) {  // FP32 Jacobi + FP64 polish in shared memory
    const size_t smem = (size_t)4 * R * R * sizeof(double);
    if (cudaFuncSetAttribute(jacobi_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return RSVD_ECUDA;
    jacobi_mixed<<<batch, kJacobiThreads, smem, st>>>(C, R, H, U, eig, status_word());
    return launch_status();
  }
  const size_t need = (size_t)2 * R * R * sizeof(double);
  const int use_smem = need <= 160 * 1024 ? 1 : 0;
  const size_t smem = use_smem ? need : 0;
  if (use_smem &&
      cudaFuncSetAttribute(jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return RSVD_ECUDA;
  jacobi_eig<<<batch, kJacobiThreads, smem, st>>>(C, A, V, R, H, U, eig, use_smem, status_word());
  return launch_status();
}

}  // namespace rsvd
