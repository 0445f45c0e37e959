"""Pins of the per-CTF construction (section 3.5): the linear identities the GPU
build relies on, and noiseless recovery through the grouped path."""

import numpy as np

import oracle as O
from synthetic import make_grouped_workload


def test_ctf_scales_the_kernel_on_both_sides():
    wl = make_grouped_workload(N=32, R=16, Q=32, N_B=6, N_A=3, G=3, snr=None, seed=1)
    C = O.radial_kernel(wl.templates, wl.grid.w)
    for g in range(3):
        Cg = O.radial_kernel(wl.ctf[g][None, :, None] * wl.templates, wl.grid.w)
        assert np.allclose(Cg, np.outer(wl.ctf[g], wl.ctf[g]) * C, rtol=0, atol=1e-13 * np.abs(Cg).max())


def test_compressing_ctf_targets_equals_compressing_with_scaled_vectors():
    wl = make_grouped_workload(N=32, R=16, Q=32, N_B=4, N_A=3, G=2, snr=None, seed=2)
    U, _ = O.grouped_principal_vectors(wl.templates, wl.grid.w, wl.ctf, 6)
    for g in range(2):
        a = O.compress(wl.ctf[g][None, :, None] * wl.templates, U[g], wl.grid.w)
        b = O.compress(wl.templates, wl.ctf[g][:, None] * U[g], wl.grid.w)
        assert np.allclose(a, b, rtol=0, atol=1e-13 * np.abs(a).max())


def test_noiseless_grouped_alignment_recovers_template_and_pose():
    wl = make_grouped_workload(N=64, R=32, Q=64, N_B=5, N_A=12, G=3, snr=None, T_side=2, seed=3)
    g = wl.grid
    U, _ = O.grouped_principal_vectors(wl.templates, g.w, wl.ctf, g.R)
    X = O.grouped_scores(wl.images, wl.offsets, wl.templates, wl.ctf, U, g.w, g.k, wl.deltas)
    best, arg = O.align_best(X)
    T = wl.deltas.shape[0]
    assert np.array_equal(np.argmax(best, axis=1), wl.truth_j)
    assert np.array_equal(arg[np.arange(12), wl.truth_j], wl.truth_t * 64 + wl.truth_m)


def test_group_vectors_are_the_principal_vectors_of_the_corrected_kernel():
    """U_g diagonalises diag(ctf_g) C diag(ctf_g) (C the kernel of the uncorrected
    templates) with its eigenvalues in decreasing order: the eigenvalues equal a
    textbook symmetric eigen-solve of that matrix."""
    wl = make_grouped_workload(N=32, R=16, Q=32, N_B=6, N_A=3, G=3, snr=None, seed=4)
    C = O.radial_kernel(wl.templates, wl.grid.w)
    H = 5
    U, lam = O.grouped_principal_vectors(wl.templates, wl.grid.w, wl.ctf, H)
    for g in range(3):
        Kg = np.outer(wl.ctf[g], wl.ctf[g]) * C
        ev = np.sort(np.linalg.eigvalsh(Kg))[::-1]
        assert np.allclose(lam[g], ev, rtol=0, atol=1e-12 * ev[0])
        D = U[g].T @ Kg @ U[g]
        assert np.allclose(D, np.diag(ev[:H]), rtol=0, atol=1e-11 * ev[0])
