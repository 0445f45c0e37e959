"""Seeded synthetic volumes for volume alignment: sums of 3-D Gaussian blobs,
whose Fourier transforms are expanded exactly in spherical harmonics on a set
of frequency shells (plane-wave expansion). No alignment arithmetic here.

Conventions:
* shells k_r = r K / R (r = 1..R), K = (pi/2) N for an N^3 grid on [-1,1]^3;
  radial weights w_r = k_r^2 dk (the k^2 dk measure; w_R halved);
* spherical harmonics orthonormal on the sphere, Condon-Shortley phase:
  Y_l^m(theta, phi) = Nbar_l^m P_l^m(cos theta) e^{i m phi}, Y_l^{-m} = (-1)^m conj(Y_l^m);
* coefficients A[r][l][m + L] (zero for |m| > l), F(k_r, khat) = sum_lm A_l^m(k_r) Y_l^m(khat);
* Fourier transform F(k) = int f(x) e^{-i k.x} dx; a blob a exp(-|x-c|^2 / (2 s^2)) has
  F(k) = a (2 pi)^{3/2} s^3 exp(-s^2 k^2 / 2) e^{-i k.c}, and
  e^{-i k.c} = 4 pi sum_l (-i)^l j_l(k |c|) sum_m conj(Y_l^m(chat)) Y_l^m(khat);
* a real volume has A_l^{-m} = (-1)^{l+m} conj(A_l^m) on every shell;
* rotating a volume by R moves its blob centres to R c; R_tau = R_z(alpha) R_y(beta) R_z(gamma).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import spherical_jn


@dataclass
class ShellGrid:
    N: int
    R: int
    L: int
    K: float
    dk: float
    k: np.ndarray  # [R]
    w: np.ndarray  # [R]


def shell_grid(N: int, R: int, L: int) -> ShellGrid:
    K = 0.5 * math.pi * N
    dk = K / R
    k = dk * np.arange(1, R + 1, dtype=np.float64)
    w = k**2 * dk
    w[-1] *= 0.5
    return ShellGrid(N=N, R=R, L=L, K=K, dk=dk, k=k, w=w)


def sph_harm_all(L: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Y[..., l, m + L] for l <= L, |m| <= l (zero elsewhere), at polar angles
    theta and azimuths phi (same shape), by the normalised associated-Legendre
    recursion in FP64."""
    theta = np.asarray(theta, dtype=np.float64)
    x = np.cos(theta)
    sx = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    shape = theta.shape
    Pbar = np.zeros(shape + (L + 1, L + 1))  # [.., l, m >= 0]
    pmm = np.full(shape, 1.0 / math.sqrt(4.0 * math.pi))
    for m in range(L + 1):
        if m > 0:
            pmm = -pmm * math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * sx
        Pbar[..., m, m] = pmm
        if m + 1 <= L:
            Pbar[..., m + 1, m] = x * math.sqrt(2.0 * m + 3.0) * pmm
        for l in range(m + 2, L + 1):
            a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
            b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
            Pbar[..., l, m] = a * (x * Pbar[..., l - 1, m] - b * Pbar[..., l - 2, m])
    Y = np.zeros(shape + (L + 1, 2 * L + 1), dtype=np.complex128)
    phi = np.asarray(phi, dtype=np.float64)
    for m in range(L + 1):
        e = np.exp(1j * m * phi)
        Y[..., :, L + m] = Pbar[..., :, m] * e[..., None]
        if m > 0:
            Y[..., :, L - m] = (-1) ** m * np.conj(Y[..., :, L + m])
    return Y


@dataclass
class VolumeBlobs:
    centres: np.ndarray  # [n, B, 3]
    widths: np.ndarray  # [n, B]
    amps: np.ndarray  # [n, B]


def draw_volume_blobs(rng: np.random.Generator, n: int, n_blobs: int = 20, ball_radius: float = 0.3,
                      width_range=(0.04, 0.08), amp_range=(0.5, 1.0)) -> VolumeBlobs:
    u = rng.standard_normal((n, n_blobs, 3))
    u /= np.linalg.norm(u, axis=-1, keepdims=True)
    rad = ball_radius * rng.random((n, n_blobs)) ** (1.0 / 3.0)
    return VolumeBlobs(centres=u * rad[..., None], widths=rng.uniform(*width_range, size=(n, n_blobs)),
                       amps=rng.uniform(*amp_range, size=(n, n_blobs)))


def rotation_matrix(alpha: float, beta: float, gamma: float) -> np.ndarray:
    """R_z(alpha) R_y(beta) R_z(gamma), right-handed."""
    def rz(t):
        return np.array([[math.cos(t), -math.sin(t), 0.0], [math.sin(t), math.cos(t), 0.0], [0.0, 0.0, 1.0]])

    def ry(t):
        return np.array([[math.cos(t), 0.0, math.sin(t)], [0.0, 1.0, 0.0], [-math.sin(t), 0.0, math.cos(t)]])

    return rz(alpha) @ ry(beta) @ rz(gamma)


def blobs_sh(grid: ShellGrid, blobs: VolumeBlobs, rotations: np.ndarray | None = None) -> np.ndarray:
    """Exact spherical-harmonic coefficients [n, R, L+1, 2L+1] of each blob volume
    (optionally rotated: rotations [n, 3, 3] applied to the centres)."""
    c = blobs.centres
    if rotations is not None:
        c = np.einsum("nij,nbj->nbi", rotations, c)
    n, B, _ = c.shape
    L = grid.L
    rc = np.linalg.norm(c, axis=-1)  # [n, B]
    th = np.arccos(np.clip(c[..., 2] / np.maximum(rc, 1e-300), -1.0, 1.0))
    ph = np.arctan2(c[..., 1], c[..., 0])
    Yc = np.conj(sph_harm_all(L, th, ph))  # [n, B, L+1, 2L+1]
    ls = np.arange(L + 1)
    jl = spherical_jn(ls[None, None, None, :], grid.k[None, None, :, None] * rc[:, :, None, None])  # [n,B,R,L+1]
    radial = (blobs.amps[:, :, None] * (2 * math.pi) ** 1.5 * blobs.widths[:, :, None] ** 3
              * np.exp(-0.5 * blobs.widths[:, :, None] ** 2 * grid.k[None, None, :] ** 2))  # [n, B, R]
    pw = 4.0 * math.pi * (-1j) ** ls  # [L+1]
    return np.einsum("nbr,nbrl,l,nblm->nrlm", radial, jl, pw, Yc)


def real_sh_noise(rng: np.random.Generator, n: int, R: int, L: int, sigma2: np.ndarray) -> np.ndarray:
    """Complex Gaussian coefficients of real random volumes (A_l^{-m} = (-1)^{l+m}
    conj(A_l^m)), variance sigma2[n] per coefficient."""
    out = np.zeros((n, R, L + 1, 2 * L + 1), dtype=np.complex128)
    s = np.sqrt(sigma2)[:, None, None]
    for l in range(L + 1):
        for m in range(1, l + 1):
            z = (rng.standard_normal((n, R)) + 1j * rng.standard_normal((n, R))) * s[..., 0] / math.sqrt(2.0)
            out[:, :, l, L + m] = z
            out[:, :, l, L - m] = (-1) ** (l + m) * np.conj(z)
        z0 = rng.standard_normal((n, R)) * s[..., 0]
        out[:, :, l, L] = z0 if l % 2 == 0 else 1j * z0
    return out


@dataclass
class VolumeWorkload:
    grid: ShellGrid
    targets: np.ndarray  # [N_B, R, L+1, 2L+1]
    volumes: np.ndarray  # [N_A, R, L+1, 2L+1]
    betas: np.ndarray  # [n_beta] interior-angle grid
    Mp: int  # azimuthal / in-plane grid size
    truth_j: np.ndarray
    truth_a: np.ndarray  # alpha index
    truth_b: np.ndarray  # beta index
    truth_c: np.ndarray  # gamma index


def beta_grid(n_beta: int) -> np.ndarray:
    """Interior angles beta_b = pi b / (n_beta - 1), b = 0..n_beta-1."""
    return math.pi * np.arange(n_beta, dtype=np.float64) / (n_beta - 1)


def make_volume_workload(N: int, R: int, L: int, N_B: int, N_A: int, snr: float | None, n_beta: int, Mp: int,
                         seed: int = 0) -> VolumeWorkload:
    """Volume n = target j0 rotated by the grid rotation (alpha_a0, beta_b0, gamma_c0)
    (blob centres rotated analytically), plus real noise at the given SNR
    (||signal||^2 / E||noise||^2 with the shell weights)."""
    rng = np.random.default_rng(seed)
    grid = shell_grid(N, R, L)
    tb = draw_volume_blobs(rng, N_B)
    targets = blobs_sh(grid, tb)
    betas = beta_grid(n_beta)
    j0 = rng.integers(0, N_B, N_A)
    a0 = rng.integers(0, Mp, N_A)
    b0 = rng.integers(0, n_beta, N_A)
    c0 = rng.integers(0, Mp, N_A)
    rots = np.stack([rotation_matrix(2 * math.pi * a0[i] / Mp, betas[b0[i]], 2 * math.pi * c0[i] / Mp)
                     for i in range(N_A)])
    vb = VolumeBlobs(centres=tb.centres[j0], widths=tb.widths[j0], amps=tb.amps[j0])
    signal = blobs_sh(grid, vb, rots)
    if snr is None:
        volumes = signal
    else:
        p_sig = np.einsum("nrlm,r->n", np.abs(signal) ** 2, grid.w)
        sigma2 = p_sig / (snr * np.sum(grid.w) * (L + 1) ** 2)
        volumes = signal + real_sh_noise(rng, N_A, R, L, sigma2)
    return VolumeWorkload(grid=grid, targets=targets, volumes=volumes, betas=betas, Mp=Mp, truth_j=j0,
                          truth_a=a0, truth_b=b0, truth_c=c0)


# Volume-alignment throughput workload: shells of a 48^3 grid (K = 24 pi),
# R = 24 shells, degrees L = 24 (M = 49 orders), ranks H_C = H_D = 8,
# M = 49 interior angles, the (alpha, gamma) grid zero-padded to 64 x 64.
# 96 seeded blob volumes (noisy rotated copies of one target, the shape of a
# 96-volumes-vs-one-target comparison) are tiled to 96 per SM of a 152-SM GPU.
VOLUME_CONFIG = dict(N=48, R=24, L=24, HC=8, HD=8, n_beta=49, Mp=64, N_B=1, n_distinct=96, N_A=96 * 152, snr=0.1)
