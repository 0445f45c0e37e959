/*
 * rsvd.h -- C ABI of the GB300 (sm_103a) radial-SVD image-alignment library.
 *
 * The library scores N_A images against N_B templates over Q rotations and
 * T translations with the radial-SVD compression of Rangan, "Radial-
 * recombination for rigid rotational alignment of images and volumes"
 * (arXiv 2202.07235). Notation follows the paper: R rings k_r with radial
 * weights w_r, Q equispaced angles psi_q = 2 pi q / Q, H principal vectors.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Polar samples are complex64 (interleaved float re, im), row-major
 *   [object][r][q]: sample (r, q) is F_hat(k_r, psi_q). Inputs must be the
 *   Fourier transforms of real images, i.e. sample (r, q + Q/2) equals the
 *   conjugate of sample (r, q); the library reads only q < Q/2 and uses this
 *   symmetry for the rest.
 * - Q must be a power of two in [16, 1024]; 1 <= R <= 256; 1 <= H <= min(R, 64);
 *   1 <= T <= 64.
 * - "dev" pointers are device memory of the current CUDA device, "host"
 *   pointers are host memory read during the call. The caller allocates and
 *   owns every buffer; the library allocates no memory, with one exception:
 *   rsvd_compress (and the host-input pipelines) with RSVD_FP16X3 take a
 *   stream-ordered temporary from the stream's memory pool (see rsvd_compress).
 * - stream is a cudaStream_t (NULL = legacy default stream). Every call only
 *   enqueues work on that stream and returns; host arrays are consumed
 *   before the call returns. Outputs are valid once the stream reaches the
 *   work.
 * - Return value: RSVD_OK or a negative RSVD_E* code (see rsvd_strerror). On
 *   an argument error nothing is enqueued. Kernels never trap: a device-side
 *   check that fails records a code in a per-device status word that
 *   rsvd_status() reports.
 */
#ifndef RSVD_H
#define RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSVD_ABI_VERSION 1

enum rsvd_status_code {
  RSVD_OK = 0,
  RSVD_EINVAL = -1,        /* NULL pointer, non-positive or inconsistent size   */
  RSVD_EUNSUPPORTED = -2,  /* size outside the limits listed above              */
  RSVD_ECUDA = -3,         /* a CUDA runtime call or kernel launch failed       */
  RSVD_EDEVICE = -4,       /* a kernel's own bounds check failed (status word)  */
  RSVD_ETIMEOUT = -5,      /* a bounded device-side wait gave up (status word)  */
  RSVD_EWORKSPACE = -6,    /* workspace pointer NULL or smaller than required   */
  RSVD_ENOCONVERGE = -7    /* eigen-solver sweep limit reached (status word)    */
};

/* Operand precision of the compressed rings (the Step-1 contraction of
 * eq. image_innerproduct_pm, X_hat(q) = 2 pi sum_h conj(a_h(q)) b_h(q)):
 *   RSVD_FP32    FP32 coefficients, FP32 arithmetic (CUDA cores)
 *   RSVD_BF16    coefficients rounded to bfloat16, products summed in FP32 on
 *                the tensor cores (single pass)
 *   RSVD_FP16    the same with IEEE half precision (single pass; coefficients
 *                below 2^-14 lose precision in the half-precision subnormal range)
 *   RSVD_BF16X3  each FP32 coefficient x split as hi = rn_bf16(x),
 *                lo = rn_bf16(x - hi); the products a_hi b_hi + a_hi b_lo + a_lo b_hi
 *                summed in FP32 on the tensor cores (about 16 significand bits)
 *   RSVD_FP16X3  the same three products with IEEE half parts of the row-scaled
 *                coefficient: each operand row (object n at translation t) is
 *                scaled by 2^e, e = 14 - E where 2^(E-1) <= m < 2^E for the row's
 *                largest component magnitude m (e clamped to [-126, 126], 0 for a
 *                zero row), so its largest |x 2^e| lies in [2^13, 2^14);
 *                hi = rn_fp16(x 2^e), lo = rn_fp16(x 2^e - hi); the scores are
 *                scaled back by 2^-(e_image + e_template) before the reductions
 *                (about 22 significand bits, whatever the inputs' scale)
 * Step 2 (the transform over q) and the reductions run in FP32 for every form.
 * The four tensor-core forms support Q in {128, 256, 512}, H <= 32, T <= 64
 * (else RSVD_EUNSUPPORTED) in rsvd_compress, rsvd_pack, rsvd_align_scores and
 * rsvd_align_best; scoring with RSVD_BF16X3 or RSVD_FP16X3 at Q = 256 and 512
 * takes H <= 18 (shared memory). The gradient entry points take RSVD_FP32 only. */
enum rsvd_precision { RSVD_FP32 = 0, RSVD_BF16 = 1, RSVD_FP16 = 2, RSVD_BF16X3 = 3, RSVD_FP16X3 = 4 };

/* RSVD_ABI_VERSION of the loaded library. */
int rsvd_abi_version(void);

/* Static text for a status code (never NULL). */
const char* rsvd_strerror(int code);

/* Synchronises `stream`, then returns and clears the status word of the
 * current device: RSVD_OK, RSVD_EDEVICE, RSVD_ETIMEOUT or RSVD_ENOCONVERGE
 * (the first failure recorded since the last call), or RSVD_ECUDA if the
 * synchronisation itself failed. */
int rsvd_status(void* stream);

/* Self-test of the device-side failure path that every bounded wait of the
 * library takes: enqueues one tiny kernel whose thread waits on an mbarrier
 * that nothing arrives on, with the same clock-bounded wait the scoring
 * kernels use; after `budget_cycles` SM clock cycles (1 .. 2^31, about a
 * second at most) the wait gives up and records RSVD_ETIMEOUT in the status
 * word, and the kernel returns. A following rsvd_status(stream) then reports
 * RSVD_ETIMEOUT and clears it; the CUDA context stays usable. Returns
 * RSVD_EINVAL for a budget outside that range, else RSVD_OK / RSVD_ECUDA
 * for the launch. */
int rsvd_selftest_wait_timeout(long long budget_cycles, void* stream);

/* ------------------------------------------------------------------------
 * Precompute: ring-ring kernel C and its principal vectors.
 * Paper section 3.3, eq. (Image_simple_kern): C_{rr'} is proportional to
 * sum_{q != 0} conj(b(k_r, q)) b(k_r', q) with b the Fourier-Bessel
 * coefficients of a template; section 3.4, eq. (image_cost_and_kern): C is
 * the mean over the N_B templates. Here ring r is weighted by sqrt(w_r) and
 * the constant prefactor is dropped:
 *   C_{rr'} = (1/N_B) sum_j sum_{q != 0} Re conj(beta_j(r,q)) beta_j(r',q),
 *   beta_j(r,q) = sqrt(w_r) b_j(k_r,q),  b_j(k_r,q) = (1/Q) sum_psi B_j(k_r,psi) e^{-i q psi}.
 * Computed in FP64 on the device. Principal vectors (section 3.3) are the
 * eigenvectors of C by decreasing eigenvalue, each signed so that its
 * largest-magnitude entry is positive.
 *
 *   R, Q       grid size                      w     host double[R] radial weights
 *   templates  dev complex64 [N_B][R][Q]      N_B   >= 1
 *   H          number of vectors kept (1..R, <= 64)
 *   U          dev double [R][H] (row r, column h) -- output
 *   eig        dev double [R] eigenvalues, decreasing -- output
 *   workspace  dev, >= rsvd_build_workspace_bytes(R, Q, N_B) bytes, 256-byte aligned
 * ------------------------------------------------------------------------ */
size_t rsvd_build_workspace_bytes(int R, int Q, int N_B);
int rsvd_build_radial_svd(int R, int Q, const double* w, const void* templates, int N_B, int H,
                          double* U, double* eig, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Translation-aware form (section 5, eq. Image_single_cost_with_translations:
 * the objective averaged over the Q grid rotations and a distribution of
 * translations of each template). Its kernel, in FP64 on the device:
 *   C_{rr'} = sqrt(w_r w_r') / N_B sum_j [ S_j(r,r') Phi_{rr'} - b_j(k_r,0) b_j(k_r',0) Psi_{rr'} ]
 *   S_j(r,r') = sum_q conj(b_j(k_r,q)) b_j(k_r',q)  (all q),
 *   Phi_{rr'} = (1/Q) sum_psi sum_t p_t cos((k_r - k_r') delta_t . n(psi)),
 *   Psi_{rr'} = (1/Q) sum_psi Re conj(phi_r(psi)) phi_r'(psi),
 *   phi_r(psi) = sum_t p_t exp(-i k_r delta_t . n(psi)),  n(psi) = (cos psi, sin psi);
 * with the single translation 0 it equals the kernel of rsvd_build_radial_svd.
 * For an isotropic Gaussian translation density of deviation sigma, Phi
 * tends to the paper's E+(k_r, k_r') = exp(-sigma^2 (k_r^2 + k_r'^2) / 2) exp(k_r k_r' sigma^2).
 *   k          host double[R] ring radii
 *   deltas     host double [T][2] translations (image units), T = 1..64
 *   weights    host double [T] probabilities (normalised here; NULL = uniform), >= 0
 *   workspace  dev, >= rsvd_build_translated_workspace_bytes(R, Q, N_B) bytes, 256-byte aligned
 * Other arguments and results as rsvd_build_radial_svd. */
size_t rsvd_build_translated_workspace_bytes(int R, int Q, int N_B);
int rsvd_build_radial_svd_translated(int R, int Q, const double* k, const double* w, const void* templates,
                                     int N_B, const double* deltas, const double* weights, int T, int H,
                                     double* U, double* eig, void* workspace, size_t workspace_bytes,
                                     void* stream);

/* One kernel per CTF group (section 3.5: the targets of micrograph g are the
 * templates corrected with its contrast-transfer function, and the kernel of
 * eq. image_cost_and_kern is built for each group). For isotropic CTFs,
 * ctf_g(k_r) multiplies ring r, so C_g = diag(ctf_g) C diag(ctf_g) with C the
 * kernel of the uncorrected templates (built once, FP64); U_g = principal
 * vectors of C_g; the corrected targets of group g compress with
 *   U_targets[g] = diag(ctf_g) U_g  (rsvd_compress of the uncorrected templates),
 * the images of group g with U[g].
 *   templates  dev complex64 [N_B][R][Q], uncorrected
 *   ctf        dev double [G][R]: ctf_g(k_r)
 *   U          dev double [G][R][H]          eig  dev double [G][R], decreasing per group
 *   U_targets  dev double [G][R][H] or NULL
 *   workspace  dev, >= rsvd_build_grouped_workspace_bytes(R, Q, N_B, G) bytes, 256-byte aligned */
size_t rsvd_build_grouped_workspace_bytes(int R, int Q, int N_B, int G);
int rsvd_build_radial_svd_grouped(int R, int Q, const double* w, const void* templates, int N_B,
                                  const double* ctf, int G, int H, double* U, double* U_targets,
                                  double* eig, void* workspace, size_t workspace_bytes, void* stream);

/* Allocation-free form of rsvd_build_radial_svd (the paper has no
 * counterpart; it is a memory-management variant of the call above).
 * For callers that cannot allocate device memory: code that receives only
 * raw pointers (a plugin or callback with no allocator of its own) and
 * services that fix their device footprint at start-up. Instead of a caller
 * workspace it uses a fixed 1 MiB device array inside the library, held by
 * every GPU that loads the library until the process exits; that bounds the
 * grid to R <= 181 rings (larger R returns RSVD_EUNSUPPORTED). It allocates
 * nothing: no cudaMalloc, no cudaFree.
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) once; make that first call before any stream
 *   capture on that device.
 * - Every call uses the same array and it keeps the last call's contents:
 *   calls that overlap on the GPU (other streams, other host threads on the
 *   same device) race; serialise them.
 * - The looked-up address is kept for the life of the process: a
 *   cudaDeviceReset (or a different driver context) between calls is not
 *   supported.
 * - The fixed array holds fewer per-slice partial sums of C than a caller
 *   workspace: five template slices at R = 128 (20 CTAs for the sums, 304
 *   with a workspace), four at R = 129 (36 CTAs), one at R = 181 (9 CTAs);
 *   for large R or N_B this entry point is therefore slower than
 *   rsvd_build_radial_svd.
 * Arguments and results are those of rsvd_build_radial_svd without the
 * workspace; results agree with it to rounding (the partial sums over
 * templates are grouped differently). */
int rsvd_build_radial_svd_noalloc(int R, int Q, const double* w, const void* templates, int N_B, int H,
                                  double* U, double* eig, void* stream);

/* ------------------------------------------------------------------------
 * Compression: translated principal-image-rings in the Fourier-Bessel basis.
 * Paper section 3.2 ([u^T A](psi_q) = sum_r u_r A(k_r, psi_q) eta_r) and
 * eq. (image_innerproduct_pm); translations T_delta of section 5
 * (eq. Image_single_cost_with_translations) act as
 * (T_delta A)^(k) = A^(k) exp(-i k . delta). For each object n and
 * translation t:
 *   A_t(r, psi)  = A_n(k_r, psi) exp(-i k_r (dx_t cos psi + dy_t sin psi))
 *   a_t(h, psi)  = sum_r U[r][h] sqrt(w_r) A_t(r, psi)
 *   a_t(h, q)    = (1/Q) sum_psi a_t(h, psi) e^{-2 pi i q psi / Q},  q = 0 .. Q/2
 *
 *   k, w       host double[R]: ring radii and radial weights
 *   U          dev double [R][H] (as written by rsvd_build_radial_svd)
 *   polar      dev complex64 [N][R][Q]
 *   deltas     host double [T][2] (dx, dy) in image units ([-1,1]^2 box);
 *              NULL means T = 1 and delta = 0 (templates)
 *   out        dev, rsvd_compressed_bytes(N, T, H, Q, precision) bytes, 16-byte aligned
 *
 * Layout of `out` for RSVD_FP32: row n*T + t holds H x (Q/2) complex64 values,
 * element [row][h][s] at offset ((row*H + h)*(Q/2) + s)*8 bytes, where slot
 * s >= 1 is a_t(h, s) and slot 0 packs the two real coefficients
 * (Re a_t(h, 0), Re a_t(h, Q/2)).
 *
 * Layout of `out` for RSVD_BF16 / RSVD_FP16 / RSVD_BF16X3 / RSVD_FP16X3 (the
 * tensor-core operand form): one plane of 16-bit floats (BF16X3, FP16X3: a hi
 * plane, then a lo plane of the same size; FP16X3 then holds one float per row,
 * the factor 2^-e of row n*T + t, starting right after the lo plane). With g = Q/64 slots per group, Hp = H rounded up so
 * that K = 2*Hp*g is a multiple of 16 (and Hp even at Q = 512), IPT = 128/T
 * objects per tile and
 * tiles = ceil(N/IPT), a plane is the array
 *   [tiles][32 groups][K/8][128 lanes][8]
 * where component (re: c = 0, im: c = 1) of (object n, translation t, vector h,
 * slot s) sits at group s % 32, k = (s / 32)*2*Hp + 2*h + c, lane (n % IPT)*T + t
 * of tile n / IPT; every other element is zero. Each [tile][group] block is
 * the 128 x K K-major operand image of one tensor-core contraction.
 * rsvd_compressed_bytes returns 0 for a size or precision outside these limits.
 * RSVD_FP16X3 needs each row's largest component before its parts are rounded:
 * rsvd_compress computes the RSVD_FP32 rings into a temporary of
 * rsvd_compressed_bytes(N, T, H, Q, RSVD_FP32) bytes taken from the stream's
 * memory pool (cudaMallocAsync / cudaFreeAsync on `stream`) and packs them as
 * rsvd_pack does; it returns RSVD_ECUDA if that allocation fails.
 * ------------------------------------------------------------------------ */
size_t rsvd_compressed_bytes(int N, int T, int H, int Q, int precision);
int rsvd_compress(int R, int Q, const double* k, const double* w, const double* U, int H,
                  const void* polar, int N, const double* deltas, int T, int precision, void* out,
                  void* stream);

/* Converts compressed rings written with RSVD_FP32 (N objects, T translations)
 * into the operand form of `precision` (RSVD_BF16, RSVD_FP16, RSVD_BF16X3 or
 * RSVD_FP16X3), rounding each FP32 component (RSVD_FP16X3: each row-scaled
 * component) to nearest (ties to even). For RSVD_FP16X3 the result equals
 * rsvd_compress with that precision byte for byte. Otherwise it equals
 * rsvd_compress called with that precision on the same input byte for byte
 * when the FP32 compression runs on the CUDA cores (R Q / 2 <= 12,288 for
 * Q in {256, 512}, and every other Q); beyond that the FP32 compression
 * projects on the tensor cores (3xTF32) while the operand forms are written
 * from a CUDA-core projection, and the two agree to the forms' rounding.
 *   c32  dev, rsvd_compressed_bytes(N, T, H, Q, RSVD_FP32) bytes, 8-byte aligned
 *   out  dev, rsvd_compressed_bytes(N, T, H, Q, precision) bytes, 16-byte aligned */
int rsvd_pack(const void* c32, int N, int T, int H, int Q, int precision, void* out, void* stream);

/* ------------------------------------------------------------------------
 * Full score array (small problems). Eq. (image_innerproduct_pm):
 *   Step 1  X_hat(q) = 2 pi sum_h conj(a_h(q)) b_h(q)
 *   Step 2  X(gamma_m) = sum_{q=0}^{Q-1} e^{-i q gamma_m} X_hat(q),  gamma_m = 2 pi m / Q
 * evaluated from the half spectrum (X_hat(Q-q) = conj(X_hat(q)) for real images).
 *
 *   cA   dev compressed images, N_A objects x T translations (rsvd_compress)
 *   cB   dev compressed templates, N_B objects, T = 1
 *        (both in the layout of `precision`; see rsvd_precision for the forms)
 *   X    dev float [N_A][T][N_B][Q] -- output; X[n][t][j][m] = X(gamma_m) for
 *        image n translated by delta_t against template j
 * ------------------------------------------------------------------------ */
int rsvd_align_scores(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                      int precision, float* X, void* stream);

/* ------------------------------------------------------------------------
 * Fused best alignment and log-sum-exp (section 2.7: gamma_opt = argmax X;
 * section 2.6 likelihood marginalised over rotations and translations).
 * Same X as rsvd_align_scores, never written to memory. For each (n, j):
 *   best[n][j] = max_{t, m} X[n][t][j][m]
 *   arg[n][j]  = t*Q + m of that maximum (smallest t*Q+m among equal values)
 *   lse[n][j]  = log sum_{t, m} exp(inv_sigma2 * X[n][t][j][m])   (if lse != NULL)
 *
 *   best dev float [N_A][N_B], arg dev int32 [N_A][N_B], lse dev float [N_A][N_B] or NULL
 *
 * FP32 at Q = 256 and 512 (H <= 16) runs the warp-specialised kernel; with
 * the environment variable RSVD_ALIGN_KERNEL=fused it runs the single-role
 * fused kernel instead (the same values up to rounding; for cross-checks and
 * measurements).
 * ------------------------------------------------------------------------ */
int rsvd_align_best(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                    int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                    void* stream);

/* ------------------------------------------------------------------------
 * Log-sum-exp alignment loss and its gradient (section 2.6 likelihood with
 * the rotations, translations and templates marginalised):
 *   L[n] = log sum_{j, t, m} exp(inv_sigma2 * X[n][t][j][m])
 *
 * rsvd_lse_rows: L[n] = log sum_j exp(lse[n][j]) from the per-pair lse of
 *   rsvd_align_best.  lse dev float [N_A][N_B]; L dev float [N_A].
 *
 * rsvd_lse_backward: gradient of sum_n gL[n] L[n] with respect to the
 * compressed rings, recomputing X (never stored). With
 * P(m) = inv_sigma2 gL[n] exp(inv_sigma2 X(m) - L[n]) and
 * G(q) = sum_m P(m) e^{+2 pi i q m / Q}:
 *   gA[row][h][q] = 2 pi sum_j b_j(h, q) conj(G(q)),   gB[j][h][q] = 2 pi sum_{n,t} a_{n,t}(h, q) G(q)
 * (convention d/dRe + i d/dIm of the full-spectrum coefficients), written in
 * the packed slot layout of rsvd_compress (slot 0: the real q = 0 and q = Q/2
 * terms). Supports Q in {128, 256, 512} and H <= 32 (else RSVD_EUNSUPPORTED).
 *   L, gL      dev float [N_A]
 *   gA         dev, layout of cA;  gB  dev, layout of cB
 *   workspace  dev, >= rsvd_lse_backward_workspace_bytes(...) bytes, 16-byte aligned
 *              (partial template gradients, summed in a fixed order: deterministic)
 *
 * rsvd_compress_backward: adjoint of rsvd_compress with U fixed: from the
 * gradient gC with respect to the compressed rings (layout of `out` of
 * rsvd_compress) to the gradient with respect to the polar samples,
 *   gpolar dev complex64 [N][R][Q], Hermitian-paired (sample (r, q + Q/2) is the
 *   conjugate of sample (r, q)).
 * ------------------------------------------------------------------------ */
int rsvd_lse_rows(const float* lse, int N_A, int N_B, float* L, void* stream);
size_t rsvd_lse_backward_workspace_bytes(int N_A, int T, int N_B, int H, int Q);
int rsvd_lse_backward(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                      int precision, float inv_sigma2, const float* L, const float* gL, void* gA,
                      void* gB, void* workspace, size_t workspace_bytes, void* stream);
/* Same as rsvd_lse_backward, except that the template gradient of this call
 * is added to gB instead of replacing it (gA is written as before). The
 * template gradient sums over every image, so a caller that streams the
 * images through in batches (each batch with its own L and gL rows) gets the
 * whole gradient by clearing gB once and accumulating every batch into it;
 * per batch the addition is one more FP32 rounding per element. */
int rsvd_lse_backward_accumulate(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                                 int precision, float inv_sigma2, const float* L, const float* gL, void* gA,
                                 void* gB, void* workspace, size_t workspace_bytes, void* stream);
int rsvd_compress_backward(int R, int Q, const double* k, const double* w, const double* U, int H,
                           const void* gC, int N, const double* deltas, int T, int precision,
                           void* gpolar, void* stream);

/* ------------------------------------------------------------------------
 * Finer rotation grid (section 2.4, after eq. image_innerproduct: X_hat
 * zero-padded before the transform over q). The landscape on P Q angles
 * gamma = 2 pi m' / (P Q) is the trigonometric interpolant
 *   X(gamma) = sum_{|q| < Q/2} X_hat(q) e^{-i q gamma} + X_hat(Q/2) cos(Q gamma / 2),
 * which equals X(gamma_m) at the Q coarse angles (m' = P m). P in {1, 2, 4, 8},
 * P Q <= 1024, RSVD_FP32 only (else RSVD_EUNSUPPORTED); generic per-pair kernel.
 *
 * rsvd_align_scores_fine: X dev float [N_A][T][N_B][P Q].
 * rsvd_align_best_fine:   as rsvd_align_best with arg = t P Q + m'.
 * rsvd_align_best_pairs:  the same for an explicit list of K (image, template)
 *   pairs, dev int32 [K][2] (8-byte aligned); best, arg, lse dev [K]. A pair
 *   outside [0, N_A) x [0, N_B) leaves its outputs unwritten and records
 *   RSVD_EDEVICE in the status word.
 * rsvd_align_best_fine_shifted: the result of rsvd_align_best_fine (up to
 *   rounding) from P passes of rsvd_align_best (the fused kernels): the
 *   landscape at gamma_m + 2 pi p / (P Q) is the coarse landscape of the
 *   templates rotated by p/P of a grid step, b_h(q) e^{-i q 2 pi p / (P Q)} for
 *   0 < |q| < Q/2 with b_h(Q/2) scaled by cos(pi p / P). Passes merge in place
 *   (ties keep the smaller fine index; lse by log-sum-exp). P in {1, 2, 4, 8},
 *   Q and H as rsvd_align_best, RSVD_FP32 compressed rings;
 *   workspace >= rsvd_align_fine_workspace_bytes(N_A, N_B, H, Q, P, lse != NULL),
 *   256-byte aligned.
 * ------------------------------------------------------------------------ */
int rsvd_align_scores_fine(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                           int precision, float* X, void* stream);
size_t rsvd_align_fine_workspace_bytes(int N_A, int N_B, int H, int Q, int P, int want_lse);
int rsvd_align_best_fine_shifted(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                                 float inv_sigma2, float* best, int32_t* arg, float* lse, void* workspace,
                                 size_t workspace_bytes, void* stream);
int rsvd_align_best_fine(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                         int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                         void* stream);
int rsvd_align_best_pairs(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q, int P,
                          int precision, const int32_t* pairs, int K, float inv_sigma2, float* best,
                          int32_t* arg, float* lse, void* stream);

/* Candidate selection for principal-mode-marching (section 5, discussion: a
 * coarse landscape at a low rank H, then the promising candidates refined at a
 * higher rank). For each image n, the `keep` templates with the largest
 * best[n][j] (equal scores in increasing j) as pairs (n, j), written to rows
 * n*keep .. n*keep + keep - 1 of `pairs` in decreasing score.
 *   best   dev float [N_A][N_B] (e.g. from rsvd_align_best at the low rank)
 *   keep   1 .. min(N_B, 64) (else RSVD_EUNSUPPORTED)
 *   pairs  dev int32 [N_A * keep][2] -- output, for rsvd_align_best_pairs */
int rsvd_select_pairs(const float* best, int N_A, int N_B, int keep, int32_t* pairs, void* stream);

/* ------------------------------------------------------------------------
 * Volume alignment (section 4). A volume is given by its spherical-harmonic
 * coefficients on R frequency shells: complex64 [N][R][L+1][2L+1], element
 * [n][r][l][m + L] = A_l^m(k_r) (orthonormal harmonics with the Condon-Shortley
 * phase; entries with |m| > l are ignored). A rotation tau = (gamma, beta, alpha)
 * is R_z(alpha) R_y(beta) R_z(gamma) and acts on the coefficients as
 *   (R_tau A)_l^{m1} = sum_{m2} e^{-i m1 alpha} d^l_{m1 m2}(beta) e^{-i m2 gamma} A_l^{m2}
 * (section 4.2); X(tau) = <A, R_tau B> = sum_r w_r sum_{l,m} conj(A_l^m(k_r)) (R_tau B)_l^m(k_r).
 * Limits: L <= 31, R <= 256, H_C <= 16, H_D <= 8; alignment also needs the compressed pair,
 * 2 H_C (L+1)(2L+1) complex64 values, in 227 KB of shared memory (e.g. H_C <= 11 at L = 24,
 * H_C <= 8 at L = 28).
 *
 * rsvd_build_volume_svd: radial kernel (eq. Volume_simple_radial_kern, l = 0
 *   excluded, sqrt(w_r w_r') weights) and degree kernel (eq.
 *   Volume_simple_degree_kern, rows and columns l = 0 zero), averaged over the
 *   N_B targets, in FP64; U dev double [R][H_C], eigU [R]; V dev double
 *   [L+1][H_D], eigV [L+1] (principal vectors by decreasing eigenvalue, largest
 *   entry positive). w host double [R] (the k^2 dk weights).
 *   workspace >= rsvd_volume_build_workspace_bytes(R, L), 256-byte aligned.
 * rsvd_volume_tables: the principal-degree Wigner tables (eq.
 *   principal_degree_wigner) [v_d^T d]_{m1 m2}(beta_b) = sum_l V[l][d] d^l_{m1 m2}(beta_b),
 *   tables dev float [n_beta][2L+1][2L+1][8] (element [b][m1+L][m2+L][d], zero for
 *   d >= H_D), 16-byte aligned; betas host double [n_beta] (<= 256).
 * rsvd_compress_volume: principal-volume-shells (section 4.5)
 *   out[n][h][l][m + L] = sum_r U[r][h] sqrt(w_r) A_l^m(k_r), complex64 [N][H_C][L+1][2L+1].
 * rsvd_align_volumes: eq. volume_innerproduct_pm Steps 1, 1b, 2 and 3 per
 *   (volume, target) pair with the 2-D transform zero-padded to Mp x Mp
 *   (Mp in {16, 32, 64}, Mp >= 2L+1): X at alpha_a = 2 pi a / Mp, gamma_c = 2 pi c / Mp,
 *   beta_b of the tables; best[n][j] = max X, arg[n][j] = b Mp^2 + a Mp + c of that
 *   maximum (smallest among equal values). cA, cB from rsvd_compress_volume.
 * ------------------------------------------------------------------------ */
size_t rsvd_volume_build_workspace_bytes(int R, int L);
int rsvd_build_volume_svd(int R, int L, const double* w, const void* targets, int N_B, int HC, int HD,
                          double* U, double* eigU, double* V, double* eigV, void* workspace,
                          size_t workspace_bytes, void* stream);
int rsvd_volume_tables(int L, int HD, const double* V, const double* betas, int n_beta, float* tables,
                       void* stream);
int rsvd_compress_volume(int R, int L, const double* w, const double* U, int HC, const void* volumes, int N,
                         void* out, void* stream);
int rsvd_align_volumes(const void* cA, int N_A, const void* cB, int N_B, int HC, int L, const double* V, int HD,
                       const float* tables, int n_beta, int Mp, float* best, int32_t* arg, void* stream);
/* Same contract for real volumes and targets (coefficients with
 * A_l^{-m} = (-1)^{l+m} conj(A_l^m), which compression with real U keeps): the
 * Step-1 product at -m is then determined by the one at m, and half of Step 1
 * is skipped. Results agree with rsvd_align_volumes up to rounding on such
 * inputs; other inputs give the wrong scores. */
int rsvd_align_volumes_real(const void* cA, int N_A, const void* cB, int N_B, int HC, int L, const double* V, int HD,
                            const float* tables, int n_beta, int Mp, float* best, int32_t* arg, void* stream);

/* ------------------------------------------------------------------------
 * Host-input pipeline: rsvd_compress (templates, then images) and
 * rsvd_align_best over images and templates held in host memory (pinned for
 * the copies to overlap), with results written to host memory.
 *   images     host complex64 [N_A][R][Q], templates host complex64 [N_B][R][Q]
 *              (polar samples as for rsvd_compress; only psi < Q/2 of each
 *              ring is copied, the samples the compression reads);
 *   best, arg  host [N_A][N_B] (lse host [N_A][N_B] or NULL): as rsvd_align_best;
 *   chunk      images per pipeline stage (e.g. a multiple of 2 x the SM count);
 *              the first stage takes chunk / 4 (chunk >= 8) to shorten the fill;
 *   workspace  device, >= rsvd_align_host_workspace_bytes(R, Q, H, T, N_B,
 *              chunk, precision, lse != NULL), 256-byte aligned, caller-owned;
 *   stream     runs the kernels; copy_stream (a different stream) runs the
 *              copies: the copy of chunk c + 1 overlaps the work on chunk c.
 * Returns after enqueueing; `stream` waits for the last copy back, so
 * synchronising `stream` makes every result visible on the host. The host
 * buffers must stay valid until then. Same limits and precisions as
 * rsvd_compress and rsvd_align_best.
 * ------------------------------------------------------------------------ */
size_t rsvd_align_host_workspace_bytes(int R, int Q, int H, int T, int N_B, int chunk, int precision,
                                       int want_lse);
int rsvd_align_best_host(int R, int Q, const double* k, const double* w, const double* U, int H,
                         const void* images, int N_A, const double* deltas, int T, const void* templates,
                         int N_B, int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                         int chunk, void* workspace, size_t workspace_bytes, void* stream, void* copy_stream);

/* ------------------------------------------------------------------------
 * Per-CTF-group alignment (section 3.5), with U and U_targets from
 * rsvd_build_radial_svd_grouped (dev double [G][R][H] each): the images of
 * group g, rows offsets[g] .. offsets[g+1]-1 of images (dev complex64
 * [N_A][R][Q]; offsets host int [G+1], non-decreasing), are compressed with U[g]
 * and aligned against the templates (dev complex64 [N_B][R][Q]) compressed
 * with U_targets[g]; best/arg dev [N_A][N_B] as rsvd_align_best. Group g runs
 * on streams[g mod n_streams] (distinct streams, n_streams >= 1); the other
 * streams first wait for the work queued on streams[0], which waits for them
 * at the end. workspace >= rsvd_align_grouped_workspace_bytes(Q, H, T, N_B,
 * largest group, precision, n_streams), 256-byte aligned.
 * ------------------------------------------------------------------------ */
size_t rsvd_align_grouped_workspace_bytes(int Q, int H, int T, int N_B, int max_group, int precision,
                                          int n_streams);
int rsvd_align_grouped(int R, int Q, const double* k, const double* w, const double* U, const double* U_targets,
                       int H, const void* images, const int* offsets, int G, const double* deltas, int T,
                       const void* templates, int N_B, int precision, float* best, int32_t* arg, void* workspace,
                       size_t workspace_bytes, void* const* streams, int n_streams);

/* Host-input volume alignment: volumes host complex64 [N_A][R][L+1][2L+1] and
 * targets host [N_B][R][L+1][2L+1] (pinned for the copies to overlap), U, V and
 * tables on the device as for rsvd_compress_volume and rsvd_align_volumes;
 * best, arg host [N_A][N_B]. The targets are copied and compressed first, then
 * the volumes in chunks of `chunk` on copy_stream (a stream other than
 * `stream`), the copy of chunk c + 1 overlapping the work on chunk c;
 * real_volumes != 0 aligns with rsvd_align_volumes_real. Returns
 * after enqueueing; `stream` waits for the last copy back. workspace >=
 * rsvd_align_volumes_host_workspace_bytes(R, L, H_C, N_B, chunk), device,
 * 256-byte aligned. */
size_t rsvd_align_volumes_host_workspace_bytes(int R, int L, int HC, int N_B, int chunk);
int rsvd_align_volumes_host(int R, int L, const double* w, const double* U, int HC, const double* V, int HD,
                            const float* tables, int n_beta, int Mp, const void* volumes, int N_A, const void* targets,
                            int N_B, int real_volumes, float* best, int32_t* arg, int chunk, void* workspace,
                            size_t workspace_bytes, void* stream, void* copy_stream);

/* Same contract as rsvd_align_best, always on the generic per-pair kernel
 * (one CTA per (image, template), all T translations, any supported Q and H).
 * Provided so callers can cross-check the fused kernel. */
int rsvd_align_best_pairwise(const void* cA, int N_A, int T, const void* cB, int N_B, int H, int Q,
                             int precision, float inv_sigma2, float* best, int32_t* arg, float* lse,
                             void* stream);

/* ------------------------------------------------------------------------
 * Arithmetic-rate probe (no counterpart in the paper: it measures the
 * denominators of the FP32-ALU and special-function rooflines on the GPU at
 * hand). Enqueues one launch of `blocks` CTAs of 256 threads, each thread
 * running independent register-resident chains of one instruction kind for
 * `iters` iterations, and stores in *ops_out (host) the number of operations
 * the launch performs: FP32 flops for RSVD_RATE_FFMA (scalar fused
 * multiply-add, 2 flops each) and RSVD_RATE_FFMA2 (packed FP32x2 fused
 * multiply-add), base-2 exponentials (ex2.approx) for RSVD_RATE_EX2. The
 * caller times the launch on `stream` (e.g. CUDA events) and divides.
 * Reads and writes no caller memory. RSVD_EINVAL for an unknown kind or
 * blocks / iters outside 1 .. 2^20 / >= 1.
 * ------------------------------------------------------------------------ */
enum rsvd_rate_kind { RSVD_RATE_FFMA = 0, RSVD_RATE_FFMA2 = 1, RSVD_RATE_EX2 = 2 };
int rsvd_rate_probe(int kind, int blocks, int iters, double* ops_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_H */
