"""Plain FP64 restatement of the paper's image-alignment computation.

Conventions (each a reading of the paper, listed with its justification in
the design notes):

* Polar samples F[..., r, q] = F_hat(k_r, psi_q), psi_q = 2 pi q / Q,
  dpsi = 2 pi / Q; radial quadrature weights w_r for the k dk measure.
* Fourier-Bessel coefficients (section 2.3, discrete form of eq. aqk) use the
  1/(2 pi) of the continuous definition: a(k_r, q) = (1/Q) sum_q' F(k_r, psi_q')
  exp(-i q psi_q'), q taken periodically in [0, Q).
* Rotation (section 2.2, eq. rotation_definition): R_gamma F(k, psi) =
  F(k, psi - gamma); X(gamma) = <A, R_gamma B> with the conjugate on A.
* Translation (section 5, eq. Image_single_cost_with_translations names
  T_delta without a formula): (T_delta A)(x) = A(x - delta), hence
  (T_delta A)^(k) = A^(k) exp(-i k . delta); scores translate the image.
* Principal-image-rings (section 3.2) scale ring r by sqrt(w_r); the constant
  sqrt(dpsi) of eta_r is dropped so that rank H = R reproduces
  eq. image_innerproduct exactly (the 2 pi of its Step 1 is kept).
* Radial kernel (section 3.3, eq. Image_simple_kern with the sqrt(w_r w_r')
  of eq. Image_single_kern kept; section 3.4, eq. image_cost_and_kern as a
  mean over the N_B templates); its constant (2 pi)^3 / (4 sigma_hat^2) is
  dropped because it does not change the principal vectors.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import logsumexp


# ---------------------------------------------------------------------------
# Section 2.3: discrete Fourier-Bessel coefficients of each image-ring.
# ---------------------------------------------------------------------------
def fb_coefficients(F: np.ndarray) -> np.ndarray:
    """a(k_r, q) = sum_q' F(k_r, psi_q') exp(-i q psi_q') dpsi / (2 pi) over the
    last axis (trapezoidal angular quadrature, section 2.3)."""
    Q = F.shape[-1]
    return np.fft.fft(F, axis=-1) / Q


# ---------------------------------------------------------------------------
# Section 5 (translations): T_delta applied in frequency space.
# ---------------------------------------------------------------------------
def translate(F: np.ndarray, k: np.ndarray, deltas: np.ndarray) -> np.ndarray:
    """F [n, R, Q] -> [n, T, R, Q], sample (r, q) multiplied by
    exp(-i k_r (delta_x cos psi_q + delta_y sin psi_q))."""
    Q = F.shape[-1]
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]
    phase = np.exp(-1j * k[None, :, None] * proj[:, None, :])  # [T, R, Q]
    return F[:, None, :, :] * phase[None]


# ---------------------------------------------------------------------------
# Section 2.2: X(gamma) = <A_hat, R_gamma B_hat> = int A^dagger(k,psi) B(k,psi-gamma) k dk dpsi,
# discretised with the polar quadrature of section 2.3 (weights w_r dpsi) and
# evaluated by brute force at every grid angle gamma_m = 2 pi m / Q.
# ---------------------------------------------------------------------------
def scores_direct(A_t: np.ndarray, B: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A_t [nA, T, R, Q] (translated images), B [nB, R, Q] ->
    complex X [nA, T, nB, Q]; X[..., m] = sum_r w_r dpsi sum_q'
    conj(A_t(r, q')) B(r, (q' - m) mod Q)."""
    nA, T, R, Q = A_t.shape
    nB = B.shape[0]
    dpsi = 2.0 * math.pi / Q
    Aw = (np.conj(A_t) * (w[None, None, :, None] * dpsi)).reshape(nA * T, R * Q)
    X = np.empty((nA * T, nB, Q), dtype=np.complex128)
    for m in range(Q):
        Bm = np.roll(B, m, axis=-1)  # Bm[..., q'] = B[..., (q' - m) mod Q]
        X[:, :, m] = Aw @ Bm.reshape(nB, R * Q).T
    return X.reshape(nA, T, nB, Q)


# ---------------------------------------------------------------------------
# Section 2.4, eq. image_innerproduct: Step 1 then Step 2 with all R rings.
# ---------------------------------------------------------------------------
def scores_fb(A_t: np.ndarray, B: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Uncompressed Fourier-Bessel route. Step 1: X_hat(q) = 2 pi sum_r w_r
    conj(a(k_r, q)) b(k_r, q). Step 2: X(gamma_m) = sum_q exp(-i q gamma_m) X_hat(q).
    Returns complex X [nA, T, nB, Q]."""
    a = fb_coefficients(A_t)  # [nA, T, R, Q]
    b = fb_coefficients(B)  # [nB, R, Q]
    Xhat = 2.0 * math.pi * np.einsum("ntrq,r,jrq->ntjq", np.conj(a), w, b)
    return np.fft.fft(Xhat, axis=-1)


# ---------------------------------------------------------------------------
# Sections 3.3-3.4: ring-ring kernel C and its principal vectors.
# ---------------------------------------------------------------------------
def radial_kernel(B: np.ndarray, w: np.ndarray, return_complex: bool = False) -> np.ndarray:
    """C_{r r'} = (1/N_B) sum_j sum_{q != 0} conj(beta_j(r, q)) beta_j(r', q),
    beta_j(r, q) = sqrt(w_r) b_j(k_r, q) (eq. Image_simple_kern averaged over
    templates as in eq. image_cost_and_kern). Returns the real part unless
    return_complex (for real images the imaginary part vanishes)."""
    b = fb_coefficients(B)  # [nB, R, Q]
    beta = np.sqrt(w)[None, :, None] * b
    beta = beta[:, :, 1:]  # drop q = 0
    C = np.einsum("jrq,jsq->rs", np.conj(beta), beta) / B.shape[0]
    return C if return_complex else C.real


def principal_vectors(C: np.ndarray, H: int) -> tuple[np.ndarray, np.ndarray]:
    """Principal vectors u_1..u_H of the symmetric kernel C (section 3.3):
    eigenvectors in order of decreasing eigenvalue, each signed so that its
    entry of largest magnitude is positive. Returns (U [R, H], eigenvalues [R]
    in decreasing order)."""
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    V = V * sgn[None, :]
    return V[:, :H].copy(), lam


# ---------------------------------------------------------------------------
# Section 3.2 + eq. image_innerproduct_pm: principal-image-rings and the
# compressed two-step score.
# ---------------------------------------------------------------------------
def compress(F_t: np.ndarray, U: np.ndarray, w: np.ndarray) -> np.ndarray:
    """[u_h^T a](q) = sum_r U_{r h} sqrt(w_r) a(k_r, q) for every q in [0, Q).
    F_t [..., R, Q] -> [..., H, Q]."""
    a = fb_coefficients(F_t)
    Wt = U * np.sqrt(w)[:, None]  # [R, H]
    return np.einsum("rh,...rq->...hq", Wt, a)


def scores_compressed(a_c: np.ndarray, b_c: np.ndarray) -> np.ndarray:
    """eq. image_innerproduct_pm. Step 1: X_hat(q) = 2 pi sum_h conj([u_h^T a](q))
    [u_h^T b](q). Step 2: X(gamma_m) = sum_q exp(-i q gamma_m) X_hat(q).
    a_c [nA, T, H, Q], b_c [nB, H, Q] -> complex X [nA, T, nB, Q]."""
    Xhat = 2.0 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(a_c), b_c)
    return np.fft.fft(Xhat, axis=-1)


# ---------------------------------------------------------------------------
# Section 2.7 (gamma_opt = argmax X) with the translations of section 5.
# ---------------------------------------------------------------------------
def align_best(X: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """X real [nA, T, nB, Q] -> best [nA, nB] = max over (t, m) and
    arg [nA, nB] = t * Q + m of the first maximum (smallest flat index)."""
    nA, T, nB, Q = X.shape
    flat = np.transpose(X, (0, 2, 1, 3)).reshape(nA, nB, T * Q)
    arg = np.argmax(flat, axis=-1)
    best = np.take_along_axis(flat, arg[..., None], axis=-1)[..., 0]
    return best, arg


# ---------------------------------------------------------------------------
# Section 2.6 likelihood, marginalised over (gamma, delta, template): the
# log-sum-exp alignment loss L = sum_n log sum_{j,t,m} exp(X / sigma^2).
# ---------------------------------------------------------------------------
def lse_pair_partials(X: np.ndarray, inv_sigma2: float) -> np.ndarray:
    """Per (image, template): log sum_{t, m} exp(X * inv_sigma2). X [nA, T, nB, Q]."""
    return logsumexp(np.transpose(X, (0, 2, 1, 3)) * inv_sigma2, axis=(2, 3))


def lse_loss(X: np.ndarray, inv_sigma2: float) -> tuple[float, np.ndarray]:
    """Returns (sum_n L_n, L [nA]) with L_n = log sum_{j, t, m} exp(X * inv_sigma2)."""
    Ln = logsumexp(X * inv_sigma2, axis=(1, 2, 3))
    return float(Ln.sum()), Ln


def lse_loss_grad(images: np.ndarray, templates: np.ndarray, k: np.ndarray, w: np.ndarray,
                  deltas: np.ndarray, U: np.ndarray, inv_sigma2: float):
    """Loss and its gradient with respect to the polar samples of the images
    and of the templates, U held fixed. Gradients follow the convention
    G = dL/dRe + i dL/dIm. Chain, in reverse order of the forward steps:

    dL/dX = inv_sigma2 * softmax_{(j,t,m)}(X * inv_sigma2) per image;
    X(m) = Re sum_q exp(-2 pi i q m / Q) X_hat(q)
        => G_Xhat(q) = sum_m exp(+2 pi i q m / Q) dL/dX(m);
    X_hat = 2 pi sum_h conj(a_h) b_h
        => G_b_h = 2 pi sum_{n,t} a_h G_Xhat,  G_a_h = 2 pi sum_j b_h conj(G_Xhat);
    a_h(q) = sum_r U_rh sqrt(w_r) a(r, q)  => G_a(r, q) = sqrt(w_r) sum_h U_rh G_a_h(q);
    a(r, q) = (1/Q) sum_psi F(r, psi) exp(-2 pi i q psi / Q)
        => G_F(r, psi) = (1/Q) sum_q exp(+2 pi i q psi / Q) G_a(r, q);
    F_t = F * phi_t  => G_F = sum_t conj(phi_t) G_F_t.
    """
    A_t = translate(images, k, deltas)  # [nA, T, R, Q]
    a_c = compress(A_t, U, w)  # [nA, T, H, Q]
    b_c = compress(templates, U, w)  # [nB, H, Q]
    loss, _, G_ac, G_bc = lse_grad_compressed(a_c, b_c, inv_sigma2)
    G_images = compress_adjoint(G_ac, U, w, k, deltas)
    G_templates = compress_adjoint(G_bc[:, None], U, w, k, np.zeros((1, 2)))
    return loss, G_images, G_templates


def lse_grad_compressed(a_c: np.ndarray, b_c: np.ndarray, inv_sigma2: float, gL: np.ndarray | None = None):
    """Loss sum_n gL_n L_n (gL = 1 by default) and its gradient with respect to the
    compressed rings a_c [nA, T, H, Q] and b_c [nB, H, Q] (full spectrum, convention
    dL/dRe + i dL/dIm). Returns (loss, L [nA], G_ac, G_bc)."""
    Q = a_c.shape[-1]
    X = scores_compressed(a_c, b_c).real  # [nA, T, nB, Q]
    _, Ln = lse_loss(X, inv_sigma2)
    g = np.ones_like(Ln) if gL is None else np.asarray(gL, dtype=np.float64)
    P = np.exp(X * inv_sigma2 - Ln[:, None, None, None]) * (inv_sigma2 * g)[:, None, None, None]  # dL/dX
    G_Xhat = np.fft.ifft(P, axis=-1) * Q  # sum_m exp(+2 pi i q m / Q) P(m)
    G_bc = 2.0 * math.pi * np.einsum("nthq,ntjq->jhq", a_c, G_Xhat)
    G_ac = 2.0 * math.pi * np.einsum("jhq,ntjq->nthq", b_c, np.conj(G_Xhat))
    return float(np.sum(g * Ln)), Ln, G_ac, G_bc


def compress_adjoint(G_c: np.ndarray, U: np.ndarray, w: np.ndarray, k: np.ndarray, deltas: np.ndarray) -> np.ndarray:
    """Adjoint of translate-then-compress, U fixed. G_c [n, T, H, Q] (gradient with
    respect to the compressed rings, full spectrum) -> gradient with respect to the
    polar samples [n, R, Q], in the convention G = dL/dRe + i dL/dIm:
    G_a(r, q) = sqrt(w_r) sum_h U_rh G_c(h, q);  G_F_t(r, psi) = (1/Q) sum_q exp(+2 pi i q psi / Q) G_a(r, q);
    G_F(r, psi) = sum_t conj(phi_t(r, psi)) G_F_t(r, psi)."""
    Q = G_c.shape[-1]
    Wt = U * np.sqrt(w)[:, None]
    G_a = np.einsum("rh,nthq->ntrq", Wt, G_c)
    G_Ft = np.fft.ifft(G_a, axis=-1)  # (1/Q) sum_q exp(+...) G_a
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]
    phase = np.exp(-1j * k[None, :, None] * proj[:, None, :])  # [T, R, Q]
    return np.einsum("ntrq,trq->nrq", G_Ft, np.conj(phase))


# ---------------------------------------------------------------------------
# Step 1 of eq. image_innerproduct_pm with reduced-precision operands. The
# paper evaluates the contraction in full precision; these forms restate it
# with the compressed coefficients rounded before the products (as tensor
# cores take them), the products and sums exact:
#   single  X_hat(q) = 2 pi sum_h conj(rn(a_h(q))) rn(b_h(q)),  rn = bf16 or fp16
#   split   x = hi + lo, hi = rn_bf16(x), lo = rn_bf16(x - hi) (per real component);
#           X_hat(q) = 2 pi sum_h [conj(a_hi) b_hi + conj(a_hi) b_lo + conj(a_lo) b_hi]
#           (the compensated bf16x3 product of Henry, Tang & Heinecke,
#           ARITH 2019; the lo*lo term is dropped).
#   scaled split (fp16x3): the same three products with IEEE half operands after
#           a power-of-two scaling of each operand row (one object at one
#           translation): x_s = x 2^e with e = 14 - E, 2^(E-1) <= m < 2^E for the
#           row's largest component magnitude m (e = 0 for a zero row), so the
#           row's largest |x_s| lies in [2^13, 2^14); hi = rn_fp16(x_s),
#           lo = rn_fp16(x_s - hi); the operand is (hi + lo) 2^-e. Half precision
#           keeps 11 significant bits per part against bfloat16's 8, and the
#           scaling keeps the parts out of its narrow exponent range's ends.
# Only the half spectrum q = 0..Q/2 is an operand (real images: the rest is
# its conjugate), and the q = 0 and q = Q/2 coefficients enter by their real
# parts.
# ---------------------------------------------------------------------------
def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 value (8 significant bits), ties to even,
    for finite x in the normal range; returned as float64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)  # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.round(np.ldexp(m, 8)), e - 8)  # np.round: half to even


def round_fp16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest IEEE binary16 value (ties to even, subnormals kept)."""
    return np.asarray(x, dtype=np.float64).astype(np.float16).astype(np.float64)


def half_spectrum_operand(c: np.ndarray) -> np.ndarray:
    """The operand a compressed ring contributes: q = 0..Q/2 with the imaginary
    parts of q = 0 and q = Q/2 dropped, extended to q = Q/2+1..Q-1 by
    conjugation. c [..., Q] complex -> [..., Q]."""
    Q = c.shape[-1]
    h = c[..., : Q // 2 + 1].copy()
    h[..., 0] = h[..., 0].real
    h[..., Q // 2] = h[..., Q // 2].real
    return np.concatenate([h, np.conj(h[..., 1 : Q // 2][..., ::-1])], axis=-1)


def _round_complex(z: np.ndarray, rn) -> np.ndarray:
    return rn(z.real) + 1j * rn(z.imag)


def pow2_row_scale(z: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Power-of-two scaling of each operand row for the fp16x3 form: z [..., H, Q]
    (one row = the leading indices) -> (z 2^e, 2^-e) with 2^-e broadcastable
    against z, e = 14 - E where 2^(E-1) <= max |Re|, |Im| of the row < 2^E
    (e = 0 for a zero row)."""
    m = np.maximum(np.abs(z.real), np.abs(z.imag)).max(axis=(-2, -1), keepdims=True)
    _, E = np.frexp(m)
    e = np.where(m > 0, 14 - E, 0)
    return np.ldexp(z.real, e) + 1j * np.ldexp(z.imag, e), np.ldexp(1.0, -e)


def operand_terms(a_c: np.ndarray, b_c: np.ndarray, form: str) -> list[tuple[np.ndarray, np.ndarray]]:
    """The (image operand, template operand) pairs whose Step-1 products are
    summed for `form` in {"fp64", "bf16", "fp16", "bf16x3", "fp16x3"}."""
    a = half_spectrum_operand(a_c)
    b = half_spectrum_operand(b_c)
    if form == "fp64":
        return [(a, b)]
    if form in ("bf16", "fp16"):
        rn = round_bf16 if form == "bf16" else round_fp16
        return [(_round_complex(a, rn), _round_complex(b, rn))]
    if form == "bf16x3":
        a_hi, b_hi = _round_complex(a, round_bf16), _round_complex(b, round_bf16)
        a_lo, b_lo = _round_complex(a - a_hi, round_bf16), _round_complex(b - b_hi, round_bf16)
        return [(a_hi, b_hi), (a_hi, b_lo), (a_lo, b_hi)]
    if form == "fp16x3":
        (a_s, fa), (b_s, fb) = pow2_row_scale(a), pow2_row_scale(b)
        a_hi, b_hi = _round_complex(a_s, round_fp16), _round_complex(b_s, round_fp16)
        a_lo, b_lo = _round_complex(a_s - a_hi, round_fp16), _round_complex(b_s - b_hi, round_fp16)
        return [(a_hi * fa, b_hi * fb), (a_hi * fa, b_lo * fb), (a_lo * fa, b_hi * fb)]
    raise ValueError(form)


def scores_compressed_form(a_c: np.ndarray, b_c: np.ndarray, form: str) -> np.ndarray:
    """Real X [nA, T, nB, Q] of eq. image_innerproduct_pm with the operands of
    `form`: X_hat = 2 pi sum over terms of sum_h conj(A) B, X = forward DFT."""
    Xhat = sum(2.0 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(A), B) for A, B in operand_terms(a_c, b_c, form))
    return np.fft.fft(Xhat, axis=-1).real


# ---------------------------------------------------------------------------
# Section 2.4 (after eq. image_innerproduct): a finer rotation grid by
# zero-padding X_hat before the transform over q. The padded transform is the
# trigonometric interpolant of the real landscape; the Nyquist coefficient
# q = Q/2 is shared equally by q = +Q/2 and q = -Q/2 so that the interpolant is
# real and takes the values X(gamma_m) at the Q coarse angles.
# ---------------------------------------------------------------------------
def scores_fine(a_c: np.ndarray, b_c: np.ndarray, P: int) -> np.ndarray:
    """Real X [nA, T, nB, P Q] at gamma = 2 pi m' / (P Q), m' = 0..PQ-1:
    X(gamma) = sum_{|q| < Q/2} X_hat(q mod Q) e^{-i q gamma} + X_hat(Q/2) cos(Q gamma / 2),
    X_hat of Step 1 (eq. image_innerproduct_pm), evaluated as a direct sum."""
    Q = a_c.shape[-1]
    Xhat = 2.0 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(a_c), b_c)
    gamma = 2.0 * math.pi * np.arange(P * Q) / (P * Q)
    q = np.arange(-(Q // 2) + 1, Q // 2)
    E = np.exp(-1j * np.outer(q, gamma))  # [2Q/2 - 1, PQ]
    X = np.einsum("ntjq,qm->ntjm", Xhat[..., q % Q], E)
    X = X + Xhat[..., Q // 2][..., None] * np.cos(0.5 * Q * gamma)
    return X.real


# ---------------------------------------------------------------------------
# Section 5 (discussion), eq. Image_single_cost_with_translations: the
# principal vectors of the objective that averages over a distribution of
# rotations (uniform on the Q grid angles) and of translations mu_delta (here
# a weighted discrete set) of the target,
#   C(u; B) = E E' sum_psi | [u^T T_d R_g B](psi) - [u^T T_d' R_g' B](psi) |^2 ,
# is quadratic in u. With b_{d,g}(r, psi) = sqrt(w_r) B(k_r, psi - g) exp(-i k_r d.n(psi)),
#   C(u; B) = 2 Q u^T K u,  K_{rr'} = (1/Q) sum_psi Re[ E conj(b_r) b_r' - conj(E b_r) E b_r' ].
# With delta = 0 only, K is the kernel of section 3.3 (q = 0 excluded).
# ---------------------------------------------------------------------------
def radial_kernel_translated(B: np.ndarray, w: np.ndarray, k: np.ndarray, deltas: np.ndarray,
                             weights: np.ndarray | None = None) -> np.ndarray:
    """K averaged over the templates B [nB, R, Q] (mean over j as in eq.
    image_cost_and_kern), by explicit expectation over the Q rotations g of the
    grid and the translations deltas [T, 2] with probabilities `weights`."""
    nB, R, Q = B.shape
    T = deltas.shape[0]
    p = np.full(T, 1.0 / T) if weights is None else np.asarray(weights, float) / np.sum(weights)
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]
    phase = np.exp(-1j * k[None, :, None] * proj[:, None, :])  # [T, R, Q]
    eta = np.sqrt(w)
    K = np.zeros((R, R))
    for j in range(nB):
        M2 = np.zeros((R, R), dtype=complex)
        m = np.zeros((R, Q), dtype=complex)
        for g in range(Q):
            rot = np.roll(B[j], g, axis=-1)  # B(k_r, psi - gamma_g)
            for t in range(T):
                b = eta[:, None] * rot * phase[t]  # [R, Q]
                M2 += (p[t] / Q) * (np.conj(b) @ b.T)  # sum over psi
                m += (p[t] / Q) * b
        K += (M2 - np.conj(m) @ m.T).real / Q
    return K / nB


def translation_moments(k: np.ndarray, deltas: np.ndarray, weights: np.ndarray | None, Q: int):
    """Phi_{rr'} = (1/Q) sum_psi E_d exp(i (k_r - k_r') d.n(psi)) and
    Psi_{rr'} = (1/Q) sum_psi conj(phi_r(psi)) phi_r'(psi), phi_r(psi) = E_d exp(-i k_r d.n(psi)):
    the translation averages in K = sqrt(w w') [S Phi - b0 b0 Psi] (S_j: the
    Parseval sum over all q of template j, b0: its ring means)."""
    T = deltas.shape[0]
    p = np.full(T, 1.0 / T) if weights is None else np.asarray(weights, float) / np.sum(weights)
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]  # [T, Q]
    dk = k[:, None] - k[None, :]
    Phi = np.einsum("t,rstq->rs", p, np.exp(1j * dk[:, :, None, None] * proj[None, None])) / Q
    phi = np.einsum("t,rtq->rq", p, np.exp(-1j * k[:, None, None] * proj[None]))
    Psi = (np.conj(phi) @ phi.T) / Q
    return Phi, Psi


def radial_kernel_translated_factored(B: np.ndarray, w: np.ndarray, k: np.ndarray, deltas: np.ndarray,
                                      weights: np.ndarray | None = None) -> np.ndarray:
    """The same kernel as radial_kernel_translated in the factorised form
    K = sqrt(w w') Re[S Phi - m Psi] (section 5): S_{rr'} = mean_j sum_q conj(b_j(r, q)) b_j(r', q)
    over all q, m_{rr'} = mean_j conj(b_j(r, 0)) b_j(r', 0), with b the FB
    coefficients and Phi, Psi from translation_moments."""
    Phi, Psi = translation_moments(k, deltas, weights, B.shape[-1])
    b = fb_coefficients(B)
    S = np.einsum("jrq,jsq->rs", np.conj(b), b) / B.shape[0]
    m = np.einsum("jr,js->rs", np.conj(b[..., 0]), b[..., 0]) / B.shape[0]
    return np.sqrt(np.outer(w, w)) * (S * Phi - m * Psi).real


# ---------------------------------------------------------------------------
# Section 3.5: one kernel per CTF. The targets of micrograph g are the
# templates corrected with that micrograph's CTF; the kernel (eq.
# image_cost_and_kern), its principal vectors and the compressed targets are
# built per group, and the images of group g are aligned to the targets of g.
# ---------------------------------------------------------------------------
def grouped_principal_vectors(S: np.ndarray, w: np.ndarray, ctf: np.ndarray, H: int):
    """S [nB, R, Q] templates, ctf [G, R] isotropic CTFs: per group g the
    principal vectors of the kernel of the targets ctf_g x S. Returns
    (U [G, R, H], lam [G, R])."""
    Us, lams = [], []
    for g in range(ctf.shape[0]):
        U, lam = principal_vectors(radial_kernel(ctf[g][None, :, None] * S, w), H)
        Us.append(U)
        lams.append(lam)
    return np.stack(Us), np.stack(lams)


def grouped_scores(images: np.ndarray, offsets: np.ndarray, S: np.ndarray, ctf: np.ndarray, U: np.ndarray,
                   w: np.ndarray, k: np.ndarray, deltas: np.ndarray) -> np.ndarray:
    """Real X [nA, T, nB, Q]: image n of group g against the targets ctf_g x S,
    both compressed with U_g (eq. image_innerproduct_pm)."""
    out = []
    for g in range(ctf.shape[0]):
        A = images[offsets[g]:offsets[g + 1]]
        if A.shape[0] == 0:
            continue
        a = compress(translate(A, k, deltas), U[g], w)
        b = compress(ctf[g][None, :, None] * S, U[g], w)
        out.append(scores_compressed(a, b).real)
    return np.concatenate(out, axis=0)
