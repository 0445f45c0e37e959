"""Seeded synthetic cryo-EM-like images and templates on a polar Fourier grid.

What is generated (the paper's experiments use EMPIAR/EMDB data, which are
not available; these stand in for them with the same shapes):

* ``polar_grid``: the polar quadrature the method is evaluated on. An N x N
  image spans [-1, 1]^2, so the pixel spacing is 2/N and the Nyquist
  frequency is K = (pi/2) N (paper section 2.3). Rings sit at
  k_r = r * K / R for r = 1..R with trapezoidal weights w_r = k_r * dk for the
  k dk measure (the k = 0 node has zero weight; the last weight is halved).
  Angles are psi_q = 2 pi q / Q.
* ``draw_blobs`` / ``blobs_polar_ft``: each image is a sum of isotropic
  Gaussians A(x) = a exp(-|x - c|^2 / (2 s^2)) with centres uniform in a disc
  of radius 0.3, widths s in U(0.02, 0.06), amplitudes a in U(0.5, 1). Its
  Fourier transform under the paper's convention (section 2.1, eq. Ahat) is
  a 2 pi s^2 exp(-s^2 |k|^2 / 2) exp(-i k . c), evaluated exactly on the polar
  nodes. Rotating an image by gamma rotates its blob centres by +gamma;
  translating it by s adds s to every centre.
* ``hermitian_noise``: detector noise in the polar domain (section 2.5): at
  node (k_r, psi_q) a complex Gaussian of variance sigma_hat^2 / (w_r dpsi),
  with node (r, q + Q/2) the conjugate of node (r, q) so that every sample
  set is the transform of a real image.
* ``make_workload``: N_B templates and N_A images; image n is template j0
  rotated by the grid angle 2 pi m0 / Q and translated by -delta_{t0}, plus
  noise at the requested SNR = ||signal||^2 / E||noise||^2 (norms in the polar
  quadrature), so that its score peaks at (j0, m0, t0).

Random streams: numpy ``default_rng(seed)`` on the host (``make_workload``)
and ``torch.Generator`` seeded with the same seed on a device
(``make_workload_torch``, for sizes the host cannot generate quickly). The
two streams differ; each is deterministic for its seed.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class PolarGrid:
    N: int
    R: int
    Q: int
    K: float
    dk: float
    dpsi: float
    k: np.ndarray = field(repr=False)  # [R] ring radii
    w: np.ndarray = field(repr=False)  # [R] radial weights for k dk
    psi: np.ndarray = field(repr=False)  # [Q] angular nodes


def polar_grid(N: int, R: int, Q: int) -> PolarGrid:
    if N <= 0 or R <= 0 or Q <= 0:
        raise ValueError("N, R, Q must be positive")
    K = 0.5 * math.pi * N
    dk = K / R
    k = dk * np.arange(1, R + 1, dtype=np.float64)
    w = k * dk
    w[-1] *= 0.5
    psi = 2.0 * math.pi * np.arange(Q, dtype=np.float64) / Q
    return PolarGrid(N=N, R=R, Q=Q, K=K, dk=dk, dpsi=2.0 * math.pi / Q, k=k, w=w, psi=psi)


def translation_grid(N: int, side: int, spacing_px: float = 1.0) -> np.ndarray:
    """side x side translations centred on 0, spacing in pixels, returned in
    image units (1 pixel = 2/N). Row t = iy * side + ix holds (dx, dy)."""
    offs = (np.arange(side, dtype=np.float64) - 0.5 * (side - 1)) * spacing_px * (2.0 / N)
    out = np.empty((side * side, 2), dtype=np.float64)
    for iy in range(side):
        for ix in range(side):
            out[iy * side + ix] = (offs[ix], offs[iy])
    return out


@dataclass
class Blobs:
    centres: np.ndarray  # [n, B, 2]
    widths: np.ndarray  # [n, B]
    amps: np.ndarray  # [n, B]


def draw_blobs(rng: np.random.Generator, n: int, n_blobs: int = 20, disc_radius: float = 0.3,
               width_range=(0.02, 0.06), amp_range=(0.5, 1.0)) -> Blobs:
    rad = disc_radius * np.sqrt(rng.random((n, n_blobs)))
    ang = 2.0 * math.pi * rng.random((n, n_blobs))
    centres = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=-1)
    widths = rng.uniform(width_range[0], width_range[1], size=(n, n_blobs))
    amps = rng.uniform(amp_range[0], amp_range[1], size=(n, n_blobs))
    return Blobs(centres=centres, widths=widths, amps=amps)


def blobs_polar_ft(grid: PolarGrid, blobs: Blobs, rotation: np.ndarray | None = None,
                   shift: np.ndarray | None = None) -> np.ndarray:
    """Exact Fourier transform of each blob image on the polar grid.

    rotation: [n] angles (blob centres rotated by +angle); shift: [n, 2]
    added to every centre after the rotation. Returns complex128 [n, R, Q].
    """
    c = blobs.centres
    n = c.shape[0]
    if rotation is not None:
        cr, sr = np.cos(rotation)[:, None], np.sin(rotation)[:, None]
        c = np.stack([cr * c[..., 0] - sr * c[..., 1], sr * c[..., 0] + cr * c[..., 1]], axis=-1)
    if shift is not None:
        c = c + shift[:, None, :]
    # angles psi < pi are evaluated; the sample at psi + pi of a real image is
    # the conjugate (F(-k) = conj F(k)), so the pairing holds bit-exactly
    half = grid.Q // 2 if grid.Q % 2 == 0 else grid.Q
    kx = grid.k[:, None] * np.cos(grid.psi[:half])[None, :]  # [R, half]
    ky = grid.k[:, None] * np.sin(grid.psi[:half])[None, :]
    k2 = (grid.k ** 2)[:, None]
    out = np.zeros((n, grid.R, half), dtype=np.complex128)
    for b in range(c.shape[1]):
        s2 = (blobs.widths[:, b] ** 2)[:, None, None]
        amp = (blobs.amps[:, b] * 2.0 * math.pi)[:, None, None] * s2 * np.exp(-0.5 * s2 * k2[None])
        ph = kx[None] * c[:, b, 0][:, None, None] + ky[None] * c[:, b, 1][:, None, None]
        out += amp * np.exp(-1j * ph)
    if half == grid.Q:
        return out
    return np.concatenate([out, np.conj(out)], axis=-1)


def polar_norm2(grid: PolarGrid, F: np.ndarray) -> np.ndarray:
    """sum_r sum_q w_r dpsi |F|^2 over the last two axes (the polar-quadrature
    squared norm used to define the SNR)."""
    return np.einsum("...rq,r->...", np.abs(F) ** 2, grid.w) * grid.dpsi


def hermitian_noise(rng: np.random.Generator, grid: PolarGrid, sigma_hat2: np.ndarray) -> np.ndarray:
    """Complex noise [n, R, Q]; node variance sigma_hat2[n] / (w_r dpsi); node
    (r, q + Q/2) is the conjugate of node (r, q). Q must be even."""
    if grid.Q % 2:
        raise ValueError("Q must be even for Hermitian-paired noise")
    n = sigma_hat2.shape[0]
    half = grid.Q // 2
    var = sigma_hat2[:, None, None] / (grid.w[None, :, None] * grid.dpsi)
    sd = np.sqrt(0.5 * var)
    z = (rng.standard_normal((n, grid.R, half)) + 1j * rng.standard_normal((n, grid.R, half))) * sd
    return np.concatenate([z, np.conj(z)], axis=-1)


@dataclass
class Workload:
    grid: PolarGrid
    deltas: np.ndarray  # [T, 2] translations tried (image units)
    templates: np.ndarray  # [N_B, R, Q] complex
    images: np.ndarray  # [N_A, R, Q] complex
    truth_j: np.ndarray  # [N_A]
    truth_m: np.ndarray  # [N_A]
    truth_t: np.ndarray  # [N_A]
    sigma_hat2: np.ndarray  # [N_A]
    template_blobs: Blobs | None = None


# The paper's workload shapes, restated (sizes from the image-alignment
# example of section 3.5 scaled to GPU batch sizes; SNR per image).
CONFIGS = {
    # plain method, FP64, tiny: 64x64 px, 32 rings, Q=128, 16 templates, 64 images
    "tiny": dict(N=64, R=32, Q=128, N_B=16, N_A=64, snr=0.1, T_side=1, H=8),
    # FP32 throughput: 128x128 px, 64 rings, Q=256, 1024 templates, 8192 images, 3x3 shifts
    "throughput": dict(N=128, R=64, Q=256, N_B=1024, N_A=8192, snr=0.05, T_side=3, H=12),
    # precision study on the tiny geometry, 256 images x 64 templates
    "precision": dict(N=64, R=32, Q=128, N_B=64, N_A=256, snr=0.1, T_side=1, H=12),
    # differentiation workload (SNR not stated; the throughput SNR is used)
    "gradient": dict(N=128, R=64, Q=256, N_B=256, N_A=4096, snr=0.05, T_side=3, H=12),
    # large throughput: 256x256 px, 128 rings, Q=512, 4096 templates, 65536 images, 5x5 shifts
    "large": dict(N=256, R=128, Q=512, N_B=4096, N_A=65536, snr=0.05, T_side=5, H=16),
}


def make_workload(N: int, R: int, Q: int, N_B: int, N_A: int, snr: float | None, T_side: int = 1,
                  seed: int = 0, spacing_px: float = 1.0, **_ignored) -> Workload:
    """Host (numpy, complex128) workload. snr=None gives noiseless images."""
    rng = np.random.default_rng(seed)
    grid = polar_grid(N, R, Q)
    deltas = translation_grid(N, T_side, spacing_px)
    T = deltas.shape[0]
    tb = draw_blobs(rng, N_B)
    templates = blobs_polar_ft(grid, tb)
    j0 = rng.integers(0, N_B, size=N_A)
    m0 = rng.integers(0, Q, size=N_A)
    t0 = rng.integers(0, T, size=N_A)
    ib = Blobs(centres=tb.centres[j0], widths=tb.widths[j0], amps=tb.amps[j0])
    signal = blobs_polar_ft(grid, ib, rotation=2.0 * math.pi * m0 / Q, shift=-deltas[t0])
    if snr is None:
        sig2 = np.zeros(N_A)
        images = signal
    else:
        sig2 = polar_norm2(grid, signal) / (snr * R * Q)
        images = signal + hermitian_noise(rng, grid, sig2)
    return Workload(grid=grid, deltas=deltas, templates=templates, images=images, truth_j=j0,
                    truth_m=m0, truth_t=t0, sigma_hat2=sig2, template_blobs=tb)


def make_workload_torch(N: int, R: int, Q: int, N_B: int, N_A: int, snr: float | None, T_side: int = 1,
                        seed: int = 0, device="cuda", spacing_px: float = 1.0, chunk: int = 512,
                        **_ignored):
    """Same construction as ``make_workload`` evaluated with torch on
    ``device`` (its own seeded stream), returned as complex64 device tensors.

    Returns (grid, deltas, templates[N_B,R,Q], images[N_A,R,Q], truth dict).
    """
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    f64 = torch.float64
    grid = polar_grid(N, R, Q)
    deltas = translation_grid(N, T_side, spacing_px)
    T = deltas.shape[0]

    def u(*shape):
        return torch.rand(*shape, generator=gen, device=device, dtype=f64)

    nb = 20
    rad = 0.3 * torch.sqrt(u(N_B, nb))
    ang = 2.0 * math.pi * u(N_B, nb)
    cen = torch.stack([rad * torch.cos(ang), rad * torch.sin(ang)], dim=-1)
    wid = 0.02 + 0.04 * u(N_B, nb)
    amp = 0.5 + 0.5 * u(N_B, nb)
    kk = torch.as_tensor(grid.k, device=device, dtype=f64)
    ps = torch.as_tensor(grid.psi, device=device, dtype=f64)
    half = Q // 2
    kx = kk[:, None] * torch.cos(ps[:half])[None, :]
    ky = kk[:, None] * torch.sin(ps[:half])[None, :]
    k2 = (kk ** 2)[:, None]
    wq = torch.as_tensor(grid.w, device=device, dtype=f64)

    def ft(c, s, a):  # c [n,B,2], s [n,B], a [n,B] -> complex128 [n,R,Q], psi+pi = conjugate
        out = torch.zeros((c.shape[0], R, half), device=device, dtype=torch.complex128)
        for b in range(c.shape[1]):
            s2 = (s[:, b] ** 2)[:, None, None]
            mag = (a[:, b] * 2.0 * math.pi)[:, None, None] * s2 * torch.exp(-0.5 * s2 * k2[None])
            ph = kx[None] * c[:, b, 0][:, None, None] + ky[None] * c[:, b, 1][:, None, None]
            out += torch.polar(mag, -ph)
        return torch.cat([out, torch.conj(out)], dim=-1)

    templates = torch.empty((N_B, R, Q), device=device, dtype=torch.complex64)
    half = Q // 2
    for i in range(0, N_B, chunk):
        templates[i:i + chunk] = ft(cen[i:i + chunk], wid[i:i + chunk], amp[i:i + chunk]).to(torch.complex64)
    j0 = torch.randint(0, N_B, (N_A,), generator=gen, device=device)
    m0 = torch.randint(0, Q, (N_A,), generator=gen, device=device)
    t0 = torch.randint(0, T, (N_A,), generator=gen, device=device)
    dl = torch.as_tensor(deltas, device=device, dtype=f64)
    images = torch.empty((N_A, R, Q), device=device, dtype=torch.complex64)
    half = Q // 2
    for i in range(0, N_A, chunk):
        jj, mm, tt = j0[i:i + chunk], m0[i:i + chunk], t0[i:i + chunk]
        g = (2.0 * math.pi / Q) * mm.to(f64)
        cr, sr = torch.cos(g)[:, None], torch.sin(g)[:, None]
        c = cen[jj]
        c = torch.stack([cr * c[..., 0] - sr * c[..., 1], sr * c[..., 0] + cr * c[..., 1]], dim=-1)
        c = c - dl[tt][:, None, :]
        sig = ft(c, wid[jj], amp[jj])
        if snr is not None:
            nrm = (sig.abs() ** 2 * wq[None, :, None]).sum(dim=(1, 2)) * grid.dpsi
            s2 = nrm / (snr * R * Q)
            var = s2[:, None, None] / (wq[None, :, None] * grid.dpsi)
            sd = torch.sqrt(0.5 * var)
            n = sig.shape[0]
            zr = torch.randn((n, R, half), generator=gen, device=device, dtype=f64)
            zi = torch.randn((n, R, half), generator=gen, device=device, dtype=f64)
            z = torch.complex(zr * sd, zi * sd)
            sig = sig + torch.cat([z, torch.conj(z)], dim=-1)
        images[i:i + chunk] = sig.to(torch.complex64)
    truth = dict(j=j0, m=m0, t=t0)
    return grid, deltas, templates, images, truth


def ctf_curves(grid: PolarGrid, G: int, seed: int = 0, amp_contrast: float = 0.1) -> np.ndarray:
    """Isotropic contrast-transfer functions standing in for G micrographs:
    ctf_g(k) = -[sqrt(1 - A^2) sin(chi_g(k)) + A cos(chi_g(k))], chi_g(k) = pi D_g (k / K)^2 * 8,
    defocus-like D_g ~ U(0.5, 1.5), amplitude contrast A. Returns float64 [G, R]."""
    rng = np.random.default_rng(seed)
    D = rng.uniform(0.5, 1.5, size=G)
    chi = math.pi * 8.0 * D[:, None] * (grid.k[None, :] / grid.K) ** 2
    return -(math.sqrt(1.0 - amp_contrast**2) * np.sin(chi) + amp_contrast * np.cos(chi))


@dataclass
class GroupedWorkload:
    grid: PolarGrid
    deltas: np.ndarray
    templates: np.ndarray  # [N_B, R, Q] before any CTF
    images: np.ndarray  # [N_A, R, Q], image n carries the CTF of its group
    ctf: np.ndarray  # [G, R]
    offsets: np.ndarray  # [G + 1]: images of group g are offsets[g] .. offsets[g+1]-1
    truth_j: np.ndarray
    truth_m: np.ndarray
    truth_t: np.ndarray


def make_grouped_workload(N: int, R: int, Q: int, N_B: int, N_A: int, G: int, snr: float | None,
                          T_side: int = 1, seed: int = 0, spacing_px: float = 1.0) -> GroupedWorkload:
    """Images in G contiguous groups (as consecutive micrographs); image n of
    group g = ctf_g x (template j0 rotated by a grid angle and translated),
    plus noise at the given SNR of that CTF-modulated signal."""
    rng = np.random.default_rng(seed)
    grid = polar_grid(N, R, Q)
    deltas = translation_grid(N, T_side, spacing_px)
    T = deltas.shape[0]
    tb = draw_blobs(rng, N_B)
    templates = blobs_polar_ft(grid, tb)
    ctf = ctf_curves(grid, G, seed + 1)
    offsets = np.round(np.linspace(0, N_A, G + 1)).astype(np.int64)
    group = np.searchsorted(offsets, np.arange(N_A), side="right") - 1
    j0 = rng.integers(0, N_B, size=N_A)
    m0 = rng.integers(0, Q, size=N_A)
    t0 = rng.integers(0, T, size=N_A)
    ib = Blobs(centres=tb.centres[j0], widths=tb.widths[j0], amps=tb.amps[j0])
    signal = blobs_polar_ft(grid, ib, rotation=2.0 * math.pi * m0 / Q, shift=-deltas[t0])
    signal = signal * ctf[group][:, :, None]
    if snr is None:
        images = signal
    else:
        sig2 = polar_norm2(grid, signal) / (snr * R * Q)
        images = signal + hermitian_noise(rng, grid, sig2)
    return GroupedWorkload(grid=grid, deltas=deltas, templates=templates, images=images, ctf=ctf, offsets=offsets,
                           truth_j=j0, truth_m=m0, truth_t=t0)
