"""Planted mistakes in the oracle functions of the finer grid (section 2.4),
the translation-aware kernel (section 5) and the per-CTF groups (section 3.5):
each mutant replaces one oracle function (on the CPU, in this process only)
with a plausible wrong variant, and the pins of that part must fail on it.
(The sign of the translation phase is not among them: the kernel averages over
the grid rotations, which include the half turn that maps delta to -delta, so
both signs give the same kernel.)"""

import math

import numpy as np
import pytest

import oracle
import oracle.rsvd_ref as R
from tests import test_oracle_grouped as pins_grouped
from tests import test_oracle_pins as pins
from tests import test_oracle_translated as pins_translated

_orig = {name: getattr(R, name) for name in
         ("scores_fine", "radial_kernel_translated", "translation_moments", "radial_kernel_translated_factored",
          "grouped_principal_vectors", "grouped_scores")}


def _fine_no_nyquist(a_c, b_c, P):
    Q = a_c.shape[-1]
    Xhat = 2.0 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(a_c), b_c)
    gamma = 2.0 * math.pi * np.arange(P * Q) / (P * Q)
    q = np.arange(-(Q // 2) + 1, Q // 2)
    return np.einsum("ntjq,qm->ntjm", Xhat[..., q % Q], np.exp(-1j * np.outer(q, gamma))).real


def _fine_wrong_sign(a_c, b_c, P):
    return _orig["scores_fine"](np.conj(a_c), np.conj(b_c), P)


def _translated_no_mean_term(B, w, k, deltas, weights=None):
    nB, Rr, Q = B.shape
    T = deltas.shape[0]
    p = np.full(T, 1.0 / T) if weights is None else np.asarray(weights, float) / np.sum(weights)
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]
    phase = np.exp(-1j * k[None, :, None] * proj[:, None, :])
    eta = np.sqrt(w)
    K = np.zeros((Rr, Rr))
    for j in range(nB):
        for g in range(Q):
            rot = np.roll(B[j], g, axis=-1)
            for t in range(T):
                b = eta[:, None] * rot * phase[t]
                K += ((p[t] / Q) * (np.conj(b) @ b.T)).real / Q
    return K / nB


def _moments_psi_unconjugated(k, deltas, weights, Q):
    Phi, _ = _orig["translation_moments"](k, deltas, weights, Q)
    T = deltas.shape[0]
    p = np.full(T, 1.0 / T) if weights is None else np.asarray(weights, float) / np.sum(weights)
    psi = 2.0 * math.pi * np.arange(Q) / Q
    proj = deltas[:, 0][:, None] * np.cos(psi)[None, :] + deltas[:, 1][:, None] * np.sin(psi)[None, :]
    phi = np.einsum("t,rtq->rq", p, np.exp(-1j * k[:, None, None] * proj[None]))
    return Phi, (phi @ phi.T) / Q


def _factored_no_mean_term(B, w, k, deltas, weights=None):
    Phi, _ = R.translation_moments(k, deltas, weights, B.shape[-1])
    b = R.fb_coefficients(B)
    S = np.einsum("jrq,jsq->rs", np.conj(b), b) / B.shape[0]
    return np.sqrt(np.outer(w, w)) * (S * Phi).real


def _grouped_ignores_ctf(S, w, ctf, H):
    U, lam = R.principal_vectors(R.radial_kernel(S, w), H)
    return np.stack([U] * ctf.shape[0]), np.stack([lam] * ctf.shape[0])


def _grouped_targets_uncorrected(images, offsets, S, ctf, U, w, k, deltas):
    out = []
    for g in range(ctf.shape[0]):
        A = images[offsets[g]:offsets[g + 1]]
        if A.shape[0] == 0:
            continue
        a = R.compress(R.translate(A, k, deltas), U[g], w)
        b = R.compress(S, U[g], w)
        out.append(R.scores_compressed(a, b).real)
    return np.concatenate(out, axis=0)


FINE_PINS = [pins.test_fine_grid_takes_the_coarse_values_at_coarse_angles,
             pins.test_fine_grid_nyquist_term_is_a_real_cosine,
             pins.test_fine_grid_matches_the_definition_at_an_off_grid_rotation,
             pins.test_finer_grid_is_coarse_landscape_of_shifted_templates]
TRANSLATED_PINS = [pins_translated.test_translation_free_kernel_is_the_section_3_kernel,
                   pins_translated.test_objective_by_brute_force_equals_its_quadratic_form,
                   pins_translated.test_factorised_kernel_equals_the_definition,
                   pins_translated.test_gaussian_translations_give_the_papers_E_plus,
                   pins_translated.test_symmetric_translation_sets_give_real_moments]
GROUPED_PINS = [pins_grouped.test_ctf_scales_the_kernel_on_both_sides,
                pins_grouped.test_compressing_ctf_targets_equals_compressing_with_scaled_vectors,
                pins_grouped.test_noiseless_grouped_alignment_recovers_template_and_pose,
                pins_grouped.test_group_vectors_are_the_principal_vectors_of_the_corrected_kernel]

MUTANTS = [
    ("scores_fine", _fine_no_nyquist, FINE_PINS),
    ("scores_fine", _fine_wrong_sign, FINE_PINS),
    ("radial_kernel_translated", _translated_no_mean_term, TRANSLATED_PINS),
    ("translation_moments", _moments_psi_unconjugated, TRANSLATED_PINS),
    ("radial_kernel_translated_factored", _factored_no_mean_term, TRANSLATED_PINS),
    ("grouped_principal_vectors", _grouped_ignores_ctf, GROUPED_PINS),
    ("grouped_scores", _grouped_targets_uncorrected, GROUPED_PINS),
]


@pytest.mark.parametrize("name,fn,tests", MUTANTS, ids=[f"{n}:{f.__name__}" for n, f, _ in MUTANTS])
def test_row_pins_catch_planted_mistake(monkeypatch, name, fn, tests):
    monkeypatch.setattr(R, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    failed = 0
    for t in tests:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    assert failed >= 1, f"no pin caught mutant {name}:{fn.__name__}"
