"""Planted mistakes in the oracle's hand-derived gradient (the adjoint chain of
the log-sum-exp loss): each mutant replaces one function (on the CPU, in this
process only) with a plausible wrong variant, and the finite-difference or
autograd pin must fail on it."""

import math

import numpy as np
import pytest

import oracle
import oracle.rsvd_ref as R
from tests import test_oracle_grad as pins

_orig = {name: getattr(R, name) for name in ("lse_grad_compressed", "compress_adjoint")}


def _grad_forward_transform(a_c, b_c, inv_sigma2, gL=None):
    """G_Xhat by the forward transform (e^{-i...}) instead of its adjoint."""
    Q = a_c.shape[-1]
    X = R.scores_compressed(a_c, b_c).real
    _, Ln = R.lse_loss(X, inv_sigma2)
    g = np.ones_like(Ln) if gL is None else np.asarray(gL, dtype=np.float64)
    P = np.exp(X * inv_sigma2 - Ln[:, None, None, None]) * (inv_sigma2 * g)[:, None, None, None]
    G_Xhat = np.fft.fft(P, axis=-1)
    G_bc = 2.0 * math.pi * np.einsum("nthq,ntjq->jhq", a_c, G_Xhat)
    G_ac = 2.0 * math.pi * np.einsum("jhq,ntjq->nthq", b_c, np.conj(G_Xhat))
    return float(np.sum(g * Ln)), Ln, G_ac, G_bc


def _grad_image_unconjugated(a_c, b_c, inv_sigma2, gL=None):
    loss, Ln, _, G_bc = _orig["lse_grad_compressed"](a_c, b_c, inv_sigma2, gL)
    Q = a_c.shape[-1]
    X = R.scores_compressed(a_c, b_c).real
    g = np.ones_like(Ln) if gL is None else np.asarray(gL, dtype=np.float64)
    P = np.exp(X * inv_sigma2 - Ln[:, None, None, None]) * (inv_sigma2 * g)[:, None, None, None]
    G_Xhat = np.fft.ifft(P, axis=-1) * Q
    G_ac = 2.0 * math.pi * np.einsum("jhq,ntjq->nthq", b_c, G_Xhat)
    return loss, Ln, G_ac, G_bc


def _grad_template_no_two_pi(a_c, b_c, inv_sigma2, gL=None):
    loss, Ln, G_ac, G_bc = _orig["lse_grad_compressed"](a_c, b_c, inv_sigma2, gL)
    return loss, Ln, G_ac, G_bc / (2.0 * math.pi)


def _adjoint_phase_unconjugated(G_c, U, w, k, deltas):
    return _orig["compress_adjoint"](G_c, U, w, k, -deltas)


def _adjoint_forward_dft(G_c, U, w, k, deltas):
    Q = G_c.shape[-1]
    return _orig["compress_adjoint"](np.fft.fft(np.fft.fft(G_c, axis=-1), axis=-1) / Q, U, w, k, deltas)


MUTANTS = [
    ("lse_grad_compressed", _grad_forward_transform),
    ("lse_grad_compressed", _grad_image_unconjugated),
    ("lse_grad_compressed", _grad_template_no_two_pi),
    ("compress_adjoint", _adjoint_phase_unconjugated),
    ("compress_adjoint", _adjoint_forward_dft),
]

PIN_TESTS = [pins.test_gradient_matches_torch_autograd, lambda: pins.test_gradient_matches_central_differences(1.0)]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[f"{n}:{f.__name__}" for n, f in MUTANTS])
def test_gradient_pins_catch_planted_mistake(monkeypatch, name, fn):
    monkeypatch.setattr(R, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    failed = 0
    for t in PIN_TESTS:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
    assert failed >= 1, f"no pin caught mutant {name}:{fn.__name__}"
