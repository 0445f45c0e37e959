"""Planted mistakes in the volume oracle (section 4): each mutant replaces one
function of oracle/volumes_ref.py (on the CPU, in this process only) with a
plausible wrong variant, and the volume pins must fail on it."""


import numpy as np
import pytest

from oracle import volumes_ref as V
from tests import test_oracle_volumes as pins

_orig = {name: getattr(V, name) for name in
         ("wigner_d", "rotate_sh", "volume_scores_fft", "_dft2", "volume_radial_kernel", "volume_degree_kernel",
          "compress_volume", "volume_scores_compressed", "volume_align_best")}


def _wigner_opposite_sense(l, beta):
    return _orig["wigner_d"](l, -beta)  # exp(+i beta J_y)


def _rotate_alpha_sign(A, alpha, beta, gamma):
    return _orig["rotate_sh"](A, -alpha, beta, gamma)


def _scores_conj_on_target(A, B, w, betas, Mp):
    return _orig["volume_scores_fft"](np.conj(A), np.conj(B), w, betas, Mp)


def _dft2_inverse(Xhat, L, Mp):
    Z = np.zeros(Xhat.shape[:-2] + (Mp, Mp), dtype=np.complex128)
    idx = np.arange(-L, L + 1) % Mp
    Z[..., idx[:, None], idx[None, :]] = Xhat
    return (np.fft.ifft2(Z, axes=(-2, -1)) * Mp * Mp).real


def _radial_keeps_l0(B, w):
    C = np.einsum("jrlm,jslm->rs", np.conj(B), B).real / B.shape[0]
    sw = np.sqrt(w)
    return C * np.outer(sw, sw)


def _degree_keeps_l0(B, w):
    return np.einsum("r,jrlm,jrkm->lk", w, np.conj(B), B).real / B.shape[0]


def _compress_no_sqrtw(A, U, w):
    return np.einsum("rh,...rlm->...hlm", U, A)


def _compressed_transposed_wigner(a, b, Vd, betas, Mp):
    L = a.shape[-2] - 1
    M = 2 * L + 1
    Xt = np.einsum("nhlx,jhly->njlxy", np.conj(a), b)
    Y = np.einsum("ld,njlxy->njdxy", Vd, Xt)
    out = np.zeros((a.shape[0], b.shape[0], len(betas), Mp, Mp))
    for bi, beta in enumerate(betas):
        vd = np.zeros((Vd.shape[1], M, M))
        for l in range(L + 1):
            s = slice(L - l, L + l + 1)
            vd[:, s, s] += Vd[l][:, None, None] * V.wigner_d(l, beta).T[None]
        out[:, :, bi] = V._dft2(np.einsum("dxy,njdxy->njxy", vd, Y), L, Mp)
    return out


def _align_last_tie(X):
    nA, nB = X.shape[:2]
    flat = X.reshape(nA, nB, -1)
    arg = flat.shape[-1] - 1 - np.argmax(flat[..., ::-1], axis=-1)
    return np.take_along_axis(flat, arg[..., None], axis=-1)[..., 0], arg


MUTANTS = [
    ("wigner_d", _wigner_opposite_sense),
    ("rotate_sh", _rotate_alpha_sign),
    ("volume_scores_fft", _scores_conj_on_target),
    ("_dft2", _dft2_inverse),
    ("volume_radial_kernel", _radial_keeps_l0),
    ("volume_degree_kernel", _degree_keeps_l0),
    ("compress_volume", _compress_no_sqrtw),
    ("volume_scores_compressed", _compressed_transposed_wigner),
    ("volume_align_best", _align_last_tie),
]

PIN_TESTS = [
    pins.test_wigner_d_closed_forms_and_group_properties,
    pins.test_rotation_of_coefficients_equals_rotating_the_blobs,
    pins.test_fft_steps_equal_the_definition,
    pins.test_full_rank_compression_reproduces_the_scores,
    pins.test_self_alignment_at_the_grid_rotation,
    pins.test_kernels_drop_the_rotation_invariant_terms,
    pins.test_wigner_d_mirror_symmetry,
    pins.test_volume_align_best_takes_the_first_maximum,
]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[f"{n}:{f.__name__}" for n, f in MUTANTS])
def test_volume_pins_catch_planted_mistake(monkeypatch, name, fn):
    monkeypatch.setattr(V, name, fn)
    failed = 0
    for t in PIN_TESTS:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    assert failed >= 1, f"no pin caught mutant {name}:{fn.__name__}"


def test_unmutated_oracle_passes_every_pin():
    for t in PIN_TESTS:
        t()
