"""Pins for the FP64 oracle: each test ties an oracle function to something
other than itself (a closed form, a brute-force evaluation of the paper's
definition, an exact identity or a textbook routine), chosen so that a dropped
term, a wrong sign or index, or a transposed operand fails at least one."""

import math

import numpy as np
import pytest
from scipy.special import jv, logsumexp

import oracle as O
from synthetic import Blobs, blobs_polar_ft, make_workload, polar_grid, polar_norm2


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --- Section 2.2 (FB coefficients as Bessel inner products): Jacobi-Anger ---
def test_fb_coefficients_match_jacobi_anger_closed_form():
    """A single Gaussian blob a exp(-|x-c|^2/(2 s^2)) has
    F(k, psi) = a 2 pi s^2 exp(-s^2 k^2 / 2) exp(-i k |c| cos(psi - theta_c)), so by
    Jacobi-Anger its FB coefficients are
    a 2 pi s^2 exp(-s^2 k^2/2) (-i)^q J_q(k |c|) exp(-i q theta_c)."""
    g = polar_grid(64, 32, 128)
    c = np.array([[[0.17, -0.11]]])
    s, amp = 0.05, 0.8
    F = blobs_polar_ft(g, Blobs(centres=c, widths=np.array([[s]]), amps=np.array([[amp]])))[0]
    a = O.fb_coefficients(F)
    rho = math.hypot(*c[0, 0])
    th = math.atan2(c[0, 0, 1], c[0, 0, 0])
    qs = np.arange(-g.Q // 2, g.Q // 2)
    env = amp * 2 * math.pi * s * s * np.exp(-0.5 * s * s * g.k ** 2)
    ref = env[:, None] * ((-1j) ** qs)[None, :] * jv(qs[None, :], g.k[:, None] * rho) * np.exp(-1j * qs * th)[None, :]
    got = a[:, qs % g.Q]
    assert _rel(got, ref) < 1e-12


# --- Section 2.2 vs section 2.4: brute-force definition == FB two-step formula ---
def test_direct_sum_equals_fourier_bessel_formula():
    wl = make_workload(N=32, R=12, Q=32, N_B=5, N_A=6, snr=0.2, T_side=3, seed=1)
    g = wl.grid
    A_t = O.translate(wl.images, g.k, wl.deltas)
    Xd = O.scores_direct(A_t, wl.templates, g.w)
    Xf = O.scores_fb(A_t, wl.templates, g.w)
    assert _rel(Xf, Xd) < 1e-12
    # real images => real landscape
    assert np.max(np.abs(Xd.imag)) < 1e-12 * np.max(np.abs(Xd.real))


# --- Sections 2.2, 2.7: exact self-alignment ---
@pytest.mark.parametrize("m0", [0, 1, 17, 127])
def test_self_alignment_scores_norm_at_the_rotation(m0):
    """Image = template rotated by the grid angle gamma_{m0} (a ring shift by m0):
    X(gamma_{m0}) = ||B||^2 in the polar quadrature, and it is the maximum."""
    wl = make_workload(N=64, R=32, Q=128, N_B=3, N_A=1, snr=None, seed=2)
    g = wl.grid
    B = wl.templates
    A = np.roll(B, m0, axis=-1)  # A(psi) = B(psi - gamma_m0)
    X = O.scores_direct(A[:, None], B, g.w).real  # [3, 1, 3, Q]
    for j in range(3):
        nrm = np.sum(g.w[:, None] * np.abs(B[j]) ** 2) * (2 * math.pi / g.Q)
        assert abs(X[j, 0, j, m0] - nrm) < 1e-12 * nrm
        assert int(np.argmax(X[j, 0, j])) == m0
    Xf = O.scores_fb(A[:, None], B, g.w).real
    assert _rel(Xf, X) < 1e-12


def test_translation_is_a_phase_matching_shifted_blob_centres():
    """(T_delta A)^ = A^ exp(-i k.delta): translating blob samples by delta equals
    the analytic transform of the blobs with centres moved by +delta."""
    g = polar_grid(64, 32, 128)
    rng = np.random.default_rng(5)
    c = rng.uniform(-0.2, 0.2, size=(2, 4, 2))
    b0 = Blobs(centres=c, widths=np.full((2, 4), 0.04), amps=np.ones((2, 4)))
    d = np.array([[0.03, -0.05]])
    moved = blobs_polar_ft(g, b0, shift=np.repeat(d, 2, axis=0))
    got = O.translate(blobs_polar_ft(g, b0), g.k, d)[:, 0]
    assert _rel(got, moved) < 1e-12


def test_noiseless_alignment_recovers_rotation_and_translation():
    """Images built as T_{-delta_t0} R_{gamma_m0} B_j0 score ||B_j0||^2 at (t0, m0)."""
    wl = make_workload(N=64, R=32, Q=128, N_B=4, N_A=12, snr=None, T_side=3, seed=3)
    g = wl.grid
    A_t = O.translate(wl.images, g.k, wl.deltas)
    X = O.scores_fb(A_t, wl.templates, g.w).real
    best, arg = O.align_best(X)
    for n in range(12):
        j = wl.truth_j[n]
        assert arg[n, j] == wl.truth_t[n] * g.Q + wl.truth_m[n]
        nrm = polar_norm2(g, wl.templates[j])
        assert abs(best[n, j] - nrm) < 1e-9 * nrm


# --- Section 3.5: H = R reproduces the full calculation to rounding ---
def test_full_rank_compression_reproduces_uncompressed_scores():
    wl = make_workload(N=64, R=32, Q=128, N_B=8, N_A=6, snr=0.1, T_side=3, seed=4)
    g = wl.grid
    C = O.radial_kernel(wl.templates, g.w)
    U, lam = O.principal_vectors(C, g.R)
    A_t = O.translate(wl.images, g.k, wl.deltas)
    Xh = O.scores_compressed(O.compress(A_t, U, g.w), O.compress(wl.templates, U, g.w))
    Xf = O.scores_fb(A_t, wl.templates, g.w)
    assert _rel(Xh, Xf) < 1e-12


def test_low_rank_compression_equals_projected_rings():
    """Rank H < R: the compressed score equals the FB formula applied to rings
    projected onto span(U) in the sqrt(w)-scaled coordinates."""
    wl = make_workload(N=64, R=32, Q=128, N_B=8, N_A=4, snr=0.1, seed=6)
    g = wl.grid
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), 8)
    P = U @ U.T
    sw = np.sqrt(g.w)

    def proj(F):  # rings -> sqrt(w)^-1 P sqrt(w) rings
        return np.einsum("rs,...sq->...rq", (P * sw[None, :]) / sw[:, None], F)

    A_t = O.translate(wl.images, g.k, wl.deltas)
    Xh = O.scores_compressed(O.compress(A_t, U, g.w), O.compress(wl.templates, U, g.w))
    Xp = O.scores_fb(proj(A_t), proj(wl.templates), g.w)
    assert _rel(Xh, Xp) < 1e-12


# --- Section 3.3: kernel C from its definition (eq. Image_single_kern) ---
def test_radial_kernel_matches_bruteforce_definition():
    """Evaluate the double rotation integral of eq. Image_single_kern on the grid
    of rotations (trapezoid in gamma, gamma'; exact here because every integrand
    frequency is below Q) and compare with the simplified eq. Image_simple_kern.
    The integral equals 2 (2 pi)^3 sum_{q != 0} conj(beta(r,q)) beta(r',q)."""
    wl = make_workload(N=16, R=6, Q=16, N_B=3, N_A=1, snr=None, seed=7)
    g = wl.grid
    sw = np.sqrt(g.w)
    Cdef = np.zeros((g.R, g.R), dtype=np.complex128)
    for B in wl.templates:
        for m in range(g.Q):
            for mp in range(g.Q):
                d = (np.roll(B, m, axis=-1) - np.roll(B, mp, axis=-1)) * sw[:, None]
                Cdef += np.conj(d) @ d.T * g.dpsi
    Cdef *= (2 * math.pi / g.Q) ** 2 / wl.templates.shape[0]
    Cdef /= 2 * (2 * math.pi) ** 3
    Cc = O.radial_kernel(wl.templates, g.w, return_complex=True)
    assert _rel(Cc, Cdef) < 1e-12
    assert np.max(np.abs(Cc.imag)) < 1e-12 * np.max(np.abs(Cc.real))


def test_radial_kernel_ignores_rotation_invariant_part():
    """A rotationally symmetric template (only q = 0 content) contributes nothing."""
    g = polar_grid(32, 16, 64)
    B = np.exp(-0.01 * g.k ** 2)[None, :, None] * np.ones((1, 1, g.Q))
    assert np.max(np.abs(O.radial_kernel(B, g.w))) < 1e-14


def test_principal_vectors_are_ordered_orthonormal_eigenvectors():
    wl = make_workload(N=64, R=32, Q=128, N_B=16, N_A=1, snr=None, seed=8)
    g = wl.grid
    C = O.radial_kernel(wl.templates, g.w)
    assert np.allclose(C, C.T, atol=1e-15 * np.abs(C).max())
    U, lam = O.principal_vectors(C, 10)
    assert np.all(np.diff(lam) <= 1e-12 * lam[0])
    assert lam[-1] > -1e-12 * lam[0]  # PSD
    assert np.allclose(U.T @ U, np.eye(10), atol=1e-12)
    assert np.allclose(C @ U, U * lam[None, :10], atol=1e-10 * lam[0])
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(10)] > 0)
    # the top vector maximises the Rayleigh quotient over random unit vectors
    rng = np.random.default_rng(0)
    v = rng.standard_normal((g.R, 200))
    v /= np.linalg.norm(v, axis=0)
    assert np.all(np.einsum("rk,rs,sk->k", v, C, v) <= lam[0] * (1 + 1e-12))
    # trace identity: tr C = mean_j sum_{q != 0} ||beta_j(q)||^2 (Parseval over psi)
    B = wl.templates
    ring_mean = B.mean(axis=-1)
    par = (np.sum(g.w[None, :, None] * np.abs(B) ** 2) / g.Q - np.sum(g.w[None] * np.abs(ring_mean) ** 2)) / B.shape[0]
    assert abs(np.trace(C) - par) < 1e-12 * par


# --- Hermitian structure of real images ---
def test_hermitian_inputs_give_hermitian_spectrum():
    wl = make_workload(N=64, R=32, Q=128, N_B=4, N_A=4, snr=0.1, T_side=3, seed=9)
    g = wl.grid
    half = g.Q // 2
    assert np.array_equal(wl.images[..., half:], np.conj(wl.images[..., :half])) or \
        _rel(wl.images[..., half:], np.conj(wl.images[..., :half])) < 1e-12
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), 12)
    a_c = O.compress(O.translate(wl.images, g.k, wl.deltas), U, g.w)
    b_c = O.compress(wl.templates, U, g.w)
    Xhat = 2 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(a_c), b_c)
    neg = Xhat[..., (-np.arange(g.Q)) % g.Q]
    assert _rel(neg, np.conj(Xhat)) < 1e-12
    X = O.scores_compressed(a_c, b_c)
    assert np.max(np.abs(X.imag)) < 1e-12 * np.max(np.abs(X.real))
    assert _rel(X.real.sum(axis=-1), g.Q * Xhat[..., 0].real) < 1e-12
    # FB coefficients of a Hermitian ring: a(-q) = (-1)^q conj(a(q)); q = 0, Q/2 real
    a = O.fb_coefficients(wl.images)
    sgn = (-1.0) ** np.arange(g.Q)
    assert _rel(a[..., (-np.arange(g.Q)) % g.Q], sgn * np.conj(a)) < 1e-12
    assert np.max(np.abs(a[..., [0, half]].imag)) < 1e-12 * np.max(np.abs(a))


# --- Section 2.1: Plancherel against a real-space closed form ---
def test_plancherel_against_real_space_gaussian_overlap():
    """X(gamma) = <A_hat, R_gamma B_hat> ~= (2 pi)^2 <A, R_gamma B>, where the
    real-space overlap of two Gaussians is a closed form. The trapezoidal radial
    rule with the zero-weight node at k = 0 integrates f(k) = k G(k) (G the
    angular integral) with the Euler-Maclaurin endpoint error
    -(dk^2 / 12) f'(0) = -(dk^2 / 12) 2 pi conj(F_A(0)) F_B(0); with that term
    added the two sides agree to the next term, (dk^4 / 720) f'''(0), which is
    below 0.3% here (without the endpoint term they differ by about 4%)."""
    g = polar_grid(128, 64, 64)
    ca, cb = np.array([0.1, 0.05]), np.array([-0.08, 0.12])
    sa, sb, aa, ab = 0.12, 0.1, 0.9, 0.7
    FA = blobs_polar_ft(g, Blobs(centres=ca[None, None], widths=np.array([[sa]]), amps=np.array([[aa]])))
    FB = blobs_polar_ft(g, Blobs(centres=cb[None, None], widths=np.array([[sb]]), amps=np.array([[ab]])))
    X = O.scores_direct(FA[:, None], FB, g.w).real[0, 0, 0]
    endpoint = (g.dk ** 2 / 12) * 2 * math.pi * (aa * 2 * math.pi * sa * sa) * (ab * 2 * math.pi * sb * sb)
    for m in range(0, g.Q, 8):
        gam = 2 * math.pi * m / g.Q
        cbr = np.array([math.cos(gam) * cb[0] - math.sin(gam) * cb[1], math.sin(gam) * cb[0] + math.cos(gam) * cb[1]])
        s2 = sa * sa + sb * sb
        ov = aa * ab * 2 * math.pi * sa * sa * sb * sb / s2 * math.exp(-np.sum((ca - cbr) ** 2) / (2 * s2))
        ref = (2 * math.pi) ** 2 * ov - endpoint
        assert abs(X[m] - ref) < 5e-3 * abs(ref)


# --- Section 2.7: argmax with the smallest-index tie rule; log-sum-exp ---
def test_align_best_matches_loops_and_breaks_ties_low():
    rng = np.random.default_rng(10)
    X = np.round(rng.standard_normal((3, 2, 4, 8)), 1)  # many exact ties
    best, arg = O.align_best(X)
    for n in range(3):
        for j in range(4):
            bv, bi = -np.inf, -1
            for t in range(2):
                for m in range(8):
                    if X[n, t, j, m] > bv:
                        bv, bi = X[n, t, j, m], t * 8 + m
            assert best[n, j] == bv and arg[n, j] == bi


def test_lse_partials_and_loss_match_definition():
    rng = np.random.default_rng(11)
    X = 3.0 * rng.standard_normal((3, 2, 4, 8))
    s = 0.7
    P = O.lse_pair_partials(X, s)
    for n in range(3):
        for j in range(4):
            assert abs(P[n, j] - math.log(np.sum(np.exp(s * X[n, :, j, :])))) < 1e-12
    loss, Ln = O.lse_loss(X, s)
    assert abs(Ln[1] - math.log(np.sum(np.exp(s * X[1])))) < 1e-12
    assert abs(loss - Ln.sum()) < 1e-12
    # the per-image loss is the log-sum-exp of the per-pair partials
    assert np.allclose(logsumexp(P, axis=1), Ln, atol=1e-12)


# ---------------------------------------------------------------------------
# Finer rotation grid by zero-padding X_hat (section 2.4).
# ---------------------------------------------------------------------------
def test_fine_grid_takes_the_coarse_values_at_coarse_angles():
    wl = make_workload(N=32, R=16, Q=32, N_B=3, N_A=4, snr=0.3, T_side=2, seed=31)
    g = wl.grid
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), 8)
    a = O.compress(O.translate(wl.images, g.k, wl.deltas), U, g.w)
    b = O.compress(wl.templates, U, g.w)
    X = O.scores_compressed(a, b).real
    for P in (1, 2, 4):
        Xf = O.scores_fine(a, b, P)
        assert Xf.shape[-1] == P * 32
        assert np.allclose(Xf[..., ::P], X, rtol=0, atol=1e-12 * np.abs(X).max())


def test_fine_grid_nyquist_term_is_a_real_cosine():
    Q, H, P = 16, 3, 4
    a = np.zeros((1, 1, H, Q), dtype=complex)
    b = np.zeros((1, H, Q), dtype=complex)
    a[..., Q // 2] = 1.0
    b[..., Q // 2] = 1.0
    gamma = 2 * math.pi * np.arange(P * Q) / (P * Q)
    ref = 2 * math.pi * H * np.cos(0.5 * Q * gamma)
    assert np.allclose(O.scores_fine(a, b, P)[0, 0, 0], ref, atol=1e-12)


def test_fine_grid_matches_the_definition_at_an_off_grid_rotation():
    """Image = template rotated analytically by a half-grid angle gamma0: the
    fine landscape's maximum sits at gamma0 and equals the direct polar-quadrature
    inner product <A, R_gamma0 B> of the definition (section 2.2)."""
    from synthetic.inputs import blobs_polar_ft, draw_blobs, polar_grid

    N, R, Q, P = 64, 32, 128, 2
    grid = polar_grid(N, R, Q)
    rng = np.random.default_rng(5)
    blobs = draw_blobs(rng, 1)
    m0 = 37
    gamma0 = 2 * math.pi * (m0 + 0.5) / Q
    B = blobs_polar_ft(grid, blobs)
    A = blobs_polar_ft(grid, blobs, rotation=np.array([gamma0]))
    U, _ = O.principal_vectors(O.radial_kernel(B, grid.w), R)
    a = O.compress(A[:, None], U, grid.w)
    b = O.compress(B, U, grid.w)
    Xf = O.scores_fine(a, b, P)[0, 0, 0]
    # definition at gamma0: <A, R_gamma0 B> with R_gamma0 B the analytically rotated template
    B_rot = blobs_polar_ft(grid, blobs, rotation=np.array([gamma0]))
    direct = float(np.real(np.sum(grid.w[:, None] * np.conj(A[0]) * B_rot[0])) * grid.dpsi)
    assert int(np.argmax(Xf)) == 2 * m0 + 1
    assert abs(Xf[2 * m0 + 1] - direct) <= 1e-8 * abs(direct)


def test_finer_grid_is_coarse_landscape_of_shifted_templates():
    """The zero-padded landscape at gamma_m + 2 pi p / (P Q) equals the coarse
    landscape of the templates rotated by p/P of a grid step in the compressed
    domain, b(q) e^{-i q 2 pi p / (P Q)} for 0 < |q| < Q/2 with the Nyquist
    coefficient scaled by cos(pi p / P): the identity the shifted GPU passes use."""
    wl = make_workload(N=32, R=8, Q=16, N_B=3, N_A=2, snr=0.3, T_side=1, seed=3)
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, wl.grid.w), 4)
    a = O.compress(O.translate(wl.images, wl.grid.k, wl.deltas), U, wl.grid.w)
    b = O.compress(wl.templates, U, wl.grid.w)
    Q = b.shape[-1]
    qs = np.where(np.arange(Q) < Q // 2, np.arange(Q), np.arange(Q) - Q)
    for P_ in (2, 3, 4):
        Xf = O.scores_fine(a, b, P_)
        for p in range(P_):
            bp = b * np.exp(-1j * qs * 2 * math.pi * p / (P_ * Q))
            bp[..., Q // 2] = b[..., Q // 2] * math.cos(math.pi * p / P_)
            Xc = O.scores_compressed(a, bp).real
            assert np.abs(Xc - Xf[..., p::P_]).max() <= 1e-12 * np.abs(Xf).max()
