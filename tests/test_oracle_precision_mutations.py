"""Planted mistakes in the oracle's reduced-precision forms: each mutant replaces
one function (on the CPU, in this process only) with a plausible wrong variant,
and the precision pins must fail on it."""

import numpy as np
import pytest

import oracle
import oracle.rsvd_ref as R
from tests import test_oracle_precision as pins

_orig = {name: getattr(R, name) for name in ("round_bf16", "half_spectrum_operand", "operand_terms", "pow2_row_scale")}


def _bf16_truncate(x):
    """Round toward zero instead of to nearest."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.trunc(np.ldexp(m, 8)), e - 8)


def _bf16_seven_bits(x):
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(np.ldexp(m, 7)), e - 7)


def _half_spectrum_keeps_imag_ends(c):
    Q = c.shape[-1]
    h = c[..., : Q // 2 + 1].copy()
    return np.concatenate([h, np.conj(h[..., 1 : Q // 2][..., ::-1])], axis=-1)


def _split_drops_cross_term(a_c, b_c, form):
    terms = _orig["operand_terms"](a_c, b_c, form)
    return terms[:2] if form == "bf16x3" else terms


def _split_lo_unrounded(a_c, b_c, form):
    if form != "bf16x3":
        return _orig["operand_terms"](a_c, b_c, form)
    a = R.half_spectrum_operand(a_c)
    b = R.half_spectrum_operand(b_c)
    rc = lambda z: R.round_bf16(z.real) + 1j * R.round_bf16(z.imag)  # noqa: E731
    a_hi, b_hi = rc(a), rc(b)
    return [(a_hi, b_hi), (a_hi, b - b_hi), (a - a_hi, b_hi)]


def _scale_one_binade_high(z):
    """Largest component in [2^14, 2^15) instead of [2^13, 2^14)."""
    zs, f = _orig["pow2_row_scale"](z)
    return zs * 2.0, f / 2.0


def _scale_factor_not_inverted(z):
    zs, f = _orig["pow2_row_scale"](z)
    return zs, 1.0 / f


def _fp16x3_unscaled(a_c, b_c, form):
    if form != "fp16x3":
        return _orig["operand_terms"](a_c, b_c, form)
    a = R.half_spectrum_operand(a_c)
    b = R.half_spectrum_operand(b_c)
    rc = lambda z: R.round_fp16(z.real) + 1j * R.round_fp16(z.imag)  # noqa: E731
    a_hi, b_hi = rc(a), rc(b)
    return [(a_hi, b_hi), (a_hi, rc(b - b_hi)), (rc(a - a_hi), b_hi)]


def _fp16x3_drops_cross_term(a_c, b_c, form):
    terms = _orig["operand_terms"](a_c, b_c, form)
    return [terms[0], terms[2]] if form == "fp16x3" else terms


def _fp16x3_lo_unrounded(a_c, b_c, form):
    if form != "fp16x3":
        return _orig["operand_terms"](a_c, b_c, form)
    (a_s, fa), (b_s, fb) = (R.pow2_row_scale(R.half_spectrum_operand(z)) for z in (a_c, b_c))
    rc = lambda z: R.round_fp16(z.real) + 1j * R.round_fp16(z.imag)  # noqa: E731
    a_hi, b_hi = rc(a_s), rc(b_s)
    return [(a_hi * fa, b_hi * fb), (a_hi * fa, (b_s - b_hi) * fb), ((a_s - a_hi) * fa, b_hi * fb)]


MUTANTS = [
    ("round_bf16", _bf16_truncate),
    ("round_bf16", _bf16_seven_bits),
    ("half_spectrum_operand", _half_spectrum_keeps_imag_ends),
    ("operand_terms", _split_drops_cross_term),
    ("operand_terms", _split_lo_unrounded),
    ("pow2_row_scale", _scale_one_binade_high),
    ("pow2_row_scale", _scale_factor_not_inverted),
    ("operand_terms", _fp16x3_unscaled),
    ("operand_terms", _fp16x3_drops_cross_term),
    ("operand_terms", _fp16x3_lo_unrounded),
]

PIN_TESTS = [getattr(pins, n) for n in dir(pins) if n.startswith("test_")]


@pytest.mark.parametrize("name,fn", MUTANTS, ids=[f"{n}:{f.__name__}" for n, f in MUTANTS])
def test_precision_pins_catch_planted_mistake(monkeypatch, name, fn):
    monkeypatch.setattr(R, name, fn)
    monkeypatch.setattr(oracle, name, fn)
    failed = 0
    for t in PIN_TESTS:
        try:
            t()
        except (AssertionError, ValueError, IndexError):
            failed += 1
        except pytest.skip.Exception:
            pass
    assert failed >= 1, f"no pin caught mutant {name}:{fn.__name__}"
