"""Plain FP64 restatement of the paper's volume alignment (section 4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Volumes are given by spherical-harmonic coefficients A[r][l][m + L] on the shells
k_r (conventions in synthetic/volumes.py). Rotations tau = (gamma, beta, alpha)
act as R_tau = R_z(alpha) R_y(beta) R_z(gamma) (section 4.1); a rotated volume
has coefficients (section 4.2)
    (R_tau A)_l^{m1} = sum_{m2} e^{-i m1 alpha} d^l_{m1 m2}(beta) e^{-i m2 gamma} A_l^{m2},
with d^l the Wigner-d matrix, here exp(-i beta J_y) in the |l, m> basis. The
inner product is X(tau) = <A, R_tau B> = sum_r w_r sum_{l,m} conj(A_l^m(k_r)) (R_tau B)_l^m(k_r).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

from .rsvd_ref import principal_vectors


def wigner_d(l: int, beta: float) -> np.ndarray:
    """d^l(beta) [m1 + l, m2 + l] = <l m1| exp(-i beta J_y) |l m2>."""
    m = np.arange(-l, l + 1, dtype=np.float64)
    jp = np.zeros((2 * l + 1, 2 * l + 1))
    for i in range(2 * l):  # J_+ |m> = sqrt(l(l+1) - m(m+1)) |m+1>
        jp[i + 1, i] = math.sqrt(l * (l + 1) - m[i] * (m[i] + 1))
    jy = (jp - jp.T) / 2j
    return expm(-1j * beta * jy).real


def rotate_sh(A: np.ndarray, alpha: float, beta: float, gamma: float) -> np.ndarray:
    """Coefficients of R_tau A, A [..., L+1, 2L+1] (section 4.2)."""
    L = A.shape[-2] - 1
    out = np.zeros_like(A, dtype=np.complex128)
    for l in range(L + 1):
        m = np.arange(-l, l + 1)
        D = np.exp(-1j * m[:, None] * alpha) * wigner_d(l, beta) * np.exp(-1j * m[None, :] * gamma)
        out[..., l, L - l:L + l + 1] = np.einsum("ab,...b->...a", D, A[..., l, L - l:L + l + 1])
    return out


def volume_scores_direct(A: np.ndarray, B: np.ndarray, w: np.ndarray, betas: np.ndarray, Mp: int) -> np.ndarray:
    """Definition: X[n, j, b, a, c] = <A_n, R_tau B_j> at tau = (gamma_c, beta_b, alpha_a),
    alpha_a = 2 pi a / Mp, gamma_c = 2 pi c / Mp, by rotating B for every tau."""
    nA, nB = A.shape[0], B.shape[0]
    X = np.zeros((nA, nB, len(betas), Mp, Mp))
    for j in range(nB):
        for b, beta in enumerate(betas):
            for a in range(Mp):
                for c in range(Mp):
                    RB = rotate_sh(B[j], 2 * math.pi * a / Mp, beta, 2 * math.pi * c / Mp)
                    X[:, j, b, a, c] = np.einsum("nrlm,rlm,r->n", np.conj(A), RB, w).real
    return X


def _dft2(Xhat: np.ndarray, L: int, Mp: int) -> np.ndarray:
    """Step 3: X(alpha_a, gamma_c) = sum_{m1,m2} e^{-i m1 alpha_a} e^{-i m2 gamma_c} Xhat(m1, m2),
    m1, m2 in [-L, L] placed periodically on an Mp x Mp grid (Mp >= 2L+1)."""
    Z = np.zeros(Xhat.shape[:-2] + (Mp, Mp), dtype=np.complex128)
    idx = np.arange(-L, L + 1) % Mp
    Z[..., idx[:, None], idx[None, :]] = Xhat
    return np.fft.fft2(Z, axes=(-2, -1)).real


def volume_scores_fft(A: np.ndarray, B: np.ndarray, w: np.ndarray, betas: np.ndarray, Mp: int) -> np.ndarray:
    """eq. volume_innerproduct: Step 1 Xt(m1, m2; l) = sum_r w_r conj(A_l^{m1}) B_l^{m2};
    Step 2 Xhat(m1, m2; beta) = sum_l d^l_{m1 m2}(beta) Xt(m1, m2; l); Step 3 the 2-D DFT."""
    L = A.shape[-2] - 1
    Xt = np.einsum("r,nrlx,jrly->njlxy", w, np.conj(A), B)
    out = np.zeros((A.shape[0], B.shape[0], len(betas), Mp, Mp))
    for b, beta in enumerate(betas):
        Xhat = np.zeros((A.shape[0], B.shape[0], 2 * L + 1, 2 * L + 1), dtype=np.complex128)
        for l in range(L + 1):
            s = slice(L - l, L + l + 1)
            Xhat[:, :, s, s] += wigner_d(l, beta)[None, None] * Xt[:, :, l, s, s]
        out[:, :, b] = _dft2(Xhat, L, Mp)
    return out


# ---------------------------------------------------------------------------
# Sections 4.5-4.9: radial and degree principal vectors, and the compressed
# Steps 1, 1b, 2, 3 (eq. volume_innerproduct_pm).
# ---------------------------------------------------------------------------
def volume_radial_kernel(B: np.ndarray, w: np.ndarray) -> np.ndarray:
    """eq. Volume_simple_radial_kern with the sqrt(w_r w_r') weights and l = 0
    excluded, averaged over the targets: C_{rr'} = sqrt(w_r w_r') / N_B sum_j
    sum_{l >= 1} sum_m Re conj(B_l^m(k_r)) B_l^m(k_r')."""
    C = np.einsum("jrlm,jslm->rs", np.conj(B[:, :, 1:]), B[:, :, 1:]).real / B.shape[0]
    sw = np.sqrt(w)
    return C * np.outer(sw, sw)


def volume_degree_kernel(B: np.ndarray, w: np.ndarray) -> np.ndarray:
    """eq. Volume_simple_degree_kern with the prefactor read as (1 - delta_{0l})(1 - delta_{0l'}):
    D_{ll'} = 1/N_B sum_j sum_r w_r sum_m Re conj(B_l^m(k_r)) B_{l'}^m(k_r), zero in row and column 0."""
    D = np.einsum("r,jrlm,jrkm->lk", w, np.conj(B), B).real / B.shape[0]
    D[0, :] = 0.0
    D[:, 0] = 0.0
    return D


def compress_volume(A: np.ndarray, U: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Principal-volume-shells (section 4.5): [u_h^T A]_l^m = sum_r U_rh sqrt(w_r) A_l^m(k_r).
    A [..., R, L+1, 2L+1] -> [..., H, L+1, 2L+1]."""
    return np.einsum("rh,...rlm->...hlm", U * np.sqrt(w)[:, None], A)


def volume_scores_compressed(a: np.ndarray, b: np.ndarray, V: np.ndarray, betas: np.ndarray, Mp: int) -> np.ndarray:
    """eq. volume_innerproduct_pm. Step 1 Xt(m1, m2; l) = sum_h conj(a_{h,l}^{m1}) b_{h,l}^{m2};
    Step 1b Y_d = sum_l V_{l d} Xt(l); Step 2 Xhat(beta) = sum_d [v_d^T d](beta) Y_d with
    [v_d^T d] = sum_l V_{l d} d^l; Step 3 the 2-D DFT. a [nA, H, L+1, M], b [nB, H, L+1, M],
    V [L+1, H_D]."""
    L = a.shape[-2] - 1
    M = 2 * L + 1
    Xt = np.einsum("nhlx,jhly->njlxy", np.conj(a), b)
    Y = np.einsum("ld,njlxy->njdxy", V, Xt)
    out = np.zeros((a.shape[0], b.shape[0], len(betas), Mp, Mp))
    for bi, beta in enumerate(betas):
        vd = np.zeros((V.shape[1], M, M))
        for l in range(L + 1):
            s = slice(L - l, L + l + 1)
            vd[:, s, s] += V[l][:, None, None] * wigner_d(l, beta)[None]
        out[:, :, bi] = _dft2(np.einsum("dxy,njdxy->njxy", vd, Y), L, Mp)
    return out


def volume_principal(K: np.ndarray, H: int):
    return principal_vectors(K, H)


def volume_align_best(X: np.ndarray):
    """X [nA, nB, n_beta, Mp, Mp] -> best [nA, nB] and arg = b Mp^2 + a Mp + c of
    the first maximum (smallest flat index)."""
    nA, nB = X.shape[:2]
    flat = X.reshape(nA, nB, -1)
    arg = np.argmax(flat, axis=-1)
    return np.take_along_axis(flat, arg[..., None], axis=-1)[..., 0], arg
