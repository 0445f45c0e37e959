"""Pins of the translation-aware ring-ring kernel (section 5, eq.
Image_single_cost_with_translations) to things other than the oracle itself:
the objective evaluated by brute force over all pairs of (rotation,
translation), the translation-free kernel of section 3.3, the paper's
Gaussian factor E+ and the factorised form the GPU evaluates."""

import math

import numpy as np

import oracle as O
from synthetic import make_workload


def _small(seed=3, Q=16, R=8, nB=2):
    wl = make_workload(N=16, R=R, Q=Q, N_B=nB, N_A=1, snr=None, T_side=2, seed=seed)
    return wl.grid, wl.templates, wl.deltas


def test_translation_free_kernel_is_the_section_3_kernel():
    g, B, _ = _small()
    K = O.radial_kernel_translated(B, g.w, g.k, np.zeros((1, 2)))
    C = O.radial_kernel(B, g.w)
    assert np.allclose(K, C, rtol=0, atol=1e-12 * np.abs(C).max())


def test_objective_by_brute_force_equals_its_quadratic_form():
    """C(u; B) = E E' sum_psi |u^T (b - b')|^2 over every pair of (rotation g,
    translation t) with probabilities p_t / Q, equals 2 Q u^T K u."""
    g, B, deltas = _small(nB=1)
    B = B[:1]
    Q, R = g.Q, g.R
    weights = np.array([0.1, 0.4, 0.3, 0.2])
    p = weights / weights.sum()
    K = O.radial_kernel_translated(B, g.w, g.k, deltas, weights)
    psi = 2 * math.pi * np.arange(Q) / Q
    eta = np.sqrt(g.w)
    states, probs = [], []
    for gg in range(Q):
        rot = np.roll(B[0], gg, axis=-1)
        for t in range(4):
            ph = np.exp(-1j * g.k[:, None] * (deltas[t, 0] * np.cos(psi) + deltas[t, 1] * np.sin(psi))[None])
            states.append(eta[:, None] * rot * ph)
            probs.append(p[t] / Q)
    S = np.array(states)  # [Q*T, R, Q]
    pr = np.array(probs)
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.standard_normal(R)
        v = np.einsum("r,srq->sq", u, S)  # u^T b for every state, every psi
        d = v[:, None, :] - v[None, :, :]
        cost = np.einsum("s,t,stq->", pr, pr, np.abs(d) ** 2)
        assert abs(cost - 2 * Q * u @ K @ u) <= 1e-10 * cost


def test_factorised_kernel_equals_the_definition():
    """K = sqrt(w w') Re[S Phi - b0 b0^T Psi] averaged over templates, with S the
    Parseval sum over all q and b0 the ring means (the form the GPU builds)."""
    g, B, deltas = _small(nB=3, Q=32, R=10, seed=8)
    # a distribution symmetric under delta -> -delta (real moments) and one that is not
    for weights in (np.array([1.0, 2.0, 2.0, 1.0]), np.array([0.1, 0.4, 0.3, 0.2])):
        K = O.radial_kernel_translated(B, g.w, g.k, deltas, weights)
        Kf = O.radial_kernel_translated_factored(B, g.w, g.k, deltas, weights)
        assert np.allclose(K, Kf, rtol=0, atol=1e-12 * np.abs(K).max())


def test_gaussian_translations_give_the_papers_E_plus():
    """An isotropic Gaussian mu_delta of standard deviation sigma (tensor
    Gauss-Hermite nodes): Phi tends to E+(k, k') = exp(-sigma^2 (k^2 + k'^2)/2) exp(k k' sigma^2)
    and Psi to exp(-sigma^2 (k^2 + k'^2)/2)."""
    sigma = 0.02
    x, wx = np.polynomial.hermite_e.hermegauss(24)  # nodes for exp(-x^2/2)
    dx, dy = np.meshgrid(sigma * x, sigma * x, indexing="ij")
    deltas = np.stack([dx.ravel(), dy.ravel()], axis=1)
    weights = np.outer(wx, wx).ravel()
    k = np.linspace(5.0, 100.0, 7)
    Phi, Psi = O.translation_moments(k, deltas, weights, 64)
    E_plus = np.exp(-0.5 * sigma**2 * (k[:, None] ** 2 + k[None, :] ** 2)) * np.exp(np.outer(k, k) * sigma**2)
    assert np.allclose(Phi, E_plus, rtol=1e-10, atol=1e-12)
    assert np.allclose(Psi, np.exp(-0.5 * sigma**2 * (k[:, None] ** 2 + k[None, :] ** 2)), rtol=1e-10, atol=1e-12)


def test_symmetric_translation_sets_give_real_moments():
    g, _, deltas = _small(Q=32, R=12)
    Phi, Psi = O.translation_moments(g.k, deltas, None, g.Q)  # 2x2 grid symmetric about 0
    assert np.max(np.abs(Phi.imag)) <= 1e-14 and np.max(np.abs(Psi.imag)) <= 1e-14
