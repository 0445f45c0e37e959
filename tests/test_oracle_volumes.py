"""Pins of the volume-alignment oracle (section 4) to things other than itself:
closed forms and group properties of the Wigner-d matrices, analytic rotation
of the blob volumes, the brute-force definition of X(tau), full-rank
equivalence of the compressed steps, and exact self-alignment."""

import math

import numpy as np

from oracle import volumes_ref as V
from synthetic.volumes import blobs_sh, draw_volume_blobs, make_volume_workload, rotation_matrix, shell_grid


def test_wigner_d_closed_forms_and_group_properties():
    b = 0.83
    d1 = V.wigner_d(1, b)
    c, s = math.cos(b), math.sin(b)
    ref = np.array([[(1 + c) / 2, s / math.sqrt(2), (1 - c) / 2],
                    [-s / math.sqrt(2), c, s / math.sqrt(2)],
                    [(1 - c) / 2, -s / math.sqrt(2), (1 + c) / 2]])  # rows m1 = -1, 0, 1
    assert np.allclose(d1, ref, atol=1e-14)
    for l in (2, 5, 9):
        d = V.wigner_d(l, b)
        assert np.allclose(d @ d.T, np.eye(2 * l + 1), atol=1e-12)
        assert np.allclose(V.wigner_d(l, 0.0), np.eye(2 * l + 1), atol=1e-14)
        assert np.allclose(V.wigner_d(l, 0.3) @ V.wigner_d(l, 0.5), V.wigner_d(l, 0.8), atol=1e-12)
        m = np.arange(-l, l + 1)
        # d^l_{m1 m2}(pi) = (-1)^{l - m2} delta_{m1, -m2}
        assert np.allclose(V.wigner_d(l, math.pi), np.diag((-1.0) ** (l - m))[::-1], atol=1e-12)


def test_rotation_of_coefficients_equals_rotating_the_blobs():
    g = shell_grid(16, 6, 14)
    rng = np.random.default_rng(2)
    blobs = draw_volume_blobs(rng, 2, n_blobs=5)
    A = blobs_sh(g, blobs)
    for al, be, ga in [(0.3, 1.2, -0.7), (2.5, 0.1, 1.9), (-1.0, 2.9, 0.4)]:
        Rm = np.stack([rotation_matrix(al, be, ga)] * 2)
        ref = blobs_sh(g, blobs, Rm)
        got = V.rotate_sh(A, al, be, ga)
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _small(seed=3, snr=0.5):
    return make_volume_workload(N=8, R=4, L=4, N_B=2, N_A=2, snr=snr, n_beta=4, Mp=10, seed=seed)


def test_fft_steps_equal_the_definition():
    wl = _small()
    Xd = V.volume_scores_direct(wl.volumes, wl.targets, wl.grid.w, wl.betas, wl.Mp)
    Xf = V.volume_scores_fft(wl.volumes, wl.targets, wl.grid.w, wl.betas, wl.Mp)
    assert np.allclose(Xf, Xd, rtol=0, atol=1e-12 * np.abs(Xd).max())


def test_scores_of_real_volumes_are_real():
    wl = _small(seed=4)
    L = wl.grid.L
    Xt = np.einsum("r,nrlx,jrly->njlxy", wl.grid.w, np.conj(wl.volumes), wl.targets)
    for beta in wl.betas:
        Xhat = np.zeros(Xt.shape[:2] + (2 * L + 1, 2 * L + 1), dtype=complex)
        for l in range(L + 1):
            s = slice(L - l, L + l + 1)
            Xhat[:, :, s, s] += V.wigner_d(l, beta) * Xt[:, :, l, s, s]
        Z = np.zeros(Xt.shape[:2] + (wl.Mp, wl.Mp), dtype=complex)
        idx = np.arange(-L, L + 1) % wl.Mp
        Z[..., idx[:, None], idx[None, :]] = Xhat
        X = np.fft.fft2(Z, axes=(-2, -1))
        assert np.abs(X.imag).max() <= 1e-12 * np.abs(X.real).max()


def test_full_rank_compression_reproduces_the_scores():
    wl = make_volume_workload(N=12, R=6, L=6, N_B=3, N_A=2, snr=0.3, n_beta=5, Mp=14, seed=5)
    g = wl.grid
    Ur, _ = V.volume_principal(V.volume_radial_kernel(wl.targets, g.w), g.R)
    Vd, _ = V.volume_principal(V.volume_degree_kernel(wl.targets, g.w), g.L + 1)
    Xf = V.volume_scores_fft(wl.volumes, wl.targets, g.w, wl.betas, wl.Mp)
    a = V.compress_volume(wl.volumes, Ur, g.w)
    b = V.compress_volume(wl.targets, Ur, g.w)
    Xc = V.volume_scores_compressed(a, b, Vd, wl.betas, wl.Mp)
    assert np.allclose(Xc, Xf, rtol=0, atol=1e-11 * np.abs(Xf).max())


def test_self_alignment_at_the_grid_rotation():
    wl = make_volume_workload(N=16, R=8, L=12, N_B=2, N_A=3, snr=None, n_beta=9, Mp=26, seed=6)
    g = wl.grid
    X = V.volume_scores_fft(wl.volumes, wl.targets, g.w, wl.betas, wl.Mp)
    best, arg = V.volume_align_best(X)
    for n in range(3):
        j = wl.truth_j[n]
        norm2 = float(np.einsum("rlm,r->", np.abs(wl.targets[j]) ** 2, g.w))
        t = wl.truth_b[n] * wl.Mp**2 + wl.truth_a[n] * wl.Mp + wl.truth_c[n]
        assert abs(X[n, j].ravel()[t] - norm2) <= 1e-10 * norm2
        assert abs(best[n, j] - norm2) <= 1e-10 * norm2


def test_kernels_drop_the_rotation_invariant_terms():
    wl = _small(seed=7, snr=None)
    g = wl.grid
    B = wl.targets.copy()
    C = V.volume_radial_kernel(B, g.w)
    D = V.volume_degree_kernel(B, g.w)
    assert np.allclose(C, C.T) and np.allclose(D, D.T)
    assert np.all(D[0] == 0) and np.all(D[:, 0] == 0)
    B0 = np.zeros_like(B)
    B0[:, :, 0] = B[:, :, 0]  # only the l = 0 (rotation-invariant) content
    assert np.abs(V.volume_radial_kernel(B0, g.w)).max() == 0.0


def test_wigner_d_mirror_symmetry():
    """d^l_{-m1,-m2}(beta) = (-1)^{m1-m2} d^l_{m1,m2}(beta): with it the GPU's Hermitian
    part of Step 1b gives Re X for any coefficients."""
    for l in (1, 4, 11):
        m = np.arange(-l, l + 1)
        for beta in (0.3, 1.7, 2.9):
            d = V.wigner_d(l, beta)
            sign = (-1.0) ** (m[:, None] - m[None, :])
            assert np.allclose(d[::-1, ::-1], sign * d, atol=1e-13)


def test_real_volumes_mirror_product():
    """For real volumes the Step-1 product at -m is (-1)^{m1-m2} conj of the one at
    m, so the Hermitian part of Step 1b is the direct product (the real-volume
    shortcut)."""
    wl = _small(seed=8)
    g = wl.grid
    L = g.L
    U = np.linalg.qr(np.random.default_rng(1).standard_normal((g.R, g.R)))[0][:, :3]
    a = V.compress_volume(wl.volumes, U, g.w)
    b = V.compress_volume(wl.targets, U, g.w)
    x = np.einsum("nhlx,jhly->njlxy", np.conj(a), b)
    m = np.arange(-L, L + 1)
    s = (-1.0) ** (m[:, None] - m[None, :])
    assert np.allclose(s * np.conj(x[..., ::-1, ::-1]), x, rtol=0, atol=1e-12 * np.abs(x).max())


def test_volume_align_best_takes_the_first_maximum():
    """max / argmax over (beta, alpha, gamma) by loops; equal maxima go to the
    smallest flat index b Mp^2 + a Mp + c."""
    rng = np.random.default_rng(9)
    X = rng.integers(0, 4, size=(2, 3, 2, 3, 3)).astype(np.float64)  # many exact ties
    best, arg = V.volume_align_best(X)
    for n in range(2):
        for j in range(3):
            bv, bi = -np.inf, -1
            for b in range(2):
                for a in range(3):
                    for c in range(3):
                        if X[n, j, b, a, c] > bv:
                            bv, bi = X[n, j, b, a, c], b * 9 + a * 3 + c
            assert best[n, j] == bv and arg[n, j] == bi
