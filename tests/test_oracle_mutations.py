"""Planted mistakes: each mutant replaces one oracle function (on the CPU, in
this process only) with a plausible wrong variant; the pin tests must fail on
it. Shows the pins constrain the arithmetic rather than restate it."""

import math

import numpy as np
import pytest

import oracle
import oracle.rsvd_ref as R
from tests import test_oracle_pins as pins

_orig = {name: getattr(R, name) for name in
         ("fb_coefficients", "translate", "radial_kernel", "principal_vectors", "compress", "scores_compressed",
          "scores_fb", "align_best")}


def _fb_wrong_sign(F):
    return np.fft.ifft(F, axis=-1)  # e^{+i q psi}


def _fb_no_norm(F):
    return np.fft.fft(F, axis=-1)


def _translate_wrong_sign(F, k, deltas):
    return np.conj(_orig["translate"](np.conj(F), k, deltas))


def _kernel_keeps_q0(B, w, return_complex=False):
    b = R.fb_coefficients(B)
    beta = np.sqrt(w)[None, :, None] * b
    C = np.einsum("jrq,jsq->rs", np.conj(beta), beta) / B.shape[0]
    return C if return_complex else C.real


def _kernel_no_weights(B, w, return_complex=False):
    return _orig["radial_kernel"](B, np.ones_like(w), return_complex)


def _compress_no_sqrtw(F_t, U, w):
    return np.einsum("rh,...rq->...hq", U, R.fb_coefficients(F_t)) * 1.0


def _scores_compressed_conj_b(a_c, b_c):
    Xhat = 2 * math.pi * np.einsum("nthq,jhq->ntjq", a_c, np.conj(b_c))
    return np.fft.fft(Xhat, axis=-1)


def _scores_fb_inverse_step2(A_t, B, w):
    a = R.fb_coefficients(A_t)
    b = R.fb_coefficients(B)
    Xhat = 2 * math.pi * np.einsum("ntrq,r,jrq->ntjq", np.conj(a), w, b)
    return np.fft.ifft(Xhat, axis=-1) * Xhat.shape[-1]


def _principal_ascending(C, H):
    lam, V = np.linalg.eigh(C)
    return V[:, :H].copy(), lam


def _align_best_last_tie(X):
    nA, T, nB, Q = X.shape
    flat = np.transpose(X, (0, 2, 1, 3)).reshape(nA, nB, T * Q)
    arg = T * Q - 1 - np.argmax(flat[..., ::-1], axis=-1)
    return np.take_along_axis(flat, arg[..., None], axis=-1)[..., 0], arg


MUTANTS = [
    ("fb_coefficients", _fb_wrong_sign),
    ("fb_coefficients", _fb_no_norm),
    ("translate", _translate_wrong_sign),
    ("radial_kernel", _kernel_keeps_q0),
    ("radial_kernel", _kernel_no_weights),
    ("compress", _compress_no_sqrtw),
    ("scores_compressed", _scores_compressed_conj_b),
    ("scores_fb", _scores_fb_inverse_step2),
    ("principal_vectors", _principal_ascending),
    ("align_best", _align_best_last_tie),
]

PIN_TESTS = [
    lambda: pins.test_fb_coefficients_match_jacobi_anger_closed_form(),
    lambda: pins.test_direct_sum_equals_fourier_bessel_formula(),
    lambda: [pins.test_self_alignment_scores_norm_at_the_rotation(m) for m in (1, 17)],
    lambda: pins.test_translation_is_a_phase_matching_shifted_blob_centres(),
    lambda: pins.test_noiseless_alignment_recovers_rotation_and_translation(),
    lambda: pins.test_full_rank_compression_reproduces_uncompressed_scores(),
    lambda: pins.test_low_rank_compression_equals_projected_rings(),
    lambda: pins.test_radial_kernel_matches_bruteforce_definition(),
    lambda: pins.test_radial_kernel_ignores_rotation_invariant_part(),
    lambda: pins.test_principal_vectors_are_ordered_orthonormal_eigenvectors(),
    lambda: pins.test_hermitian_inputs_give_hermitian_spectrum(),
    lambda: pins.test_plancherel_against_real_space_gaussian_overlap(),
    lambda: pins.test_align_best_matches_loops_and_breaks_ties_low(),
]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[f"{n}:{f.__name__}" for n, f in MUTANTS])
def test_pins_catch_planted_mistake(monkeypatch, name, fn):
    monkeypatch.setattr(R, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    monkeypatch.setattr(pins.O, name, fn)
    failed = 0
    for t in PIN_TESTS:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    assert failed >= 1, f"no pin caught mutant {name}:{fn.__name__}"
