"""Pins of the oracle's reduced-precision operand forms (the Step-1 contraction
of eq. image_innerproduct_pm with bf16 / fp16 / split-bf16x3 operands) to
things other than the oracle itself: library conversions, representability,
error bounds of the rounding, and the exact case."""

import math

import numpy as np
import pytest
import torch

import oracle as O
from synthetic import make_workload


def _scale_mix(rng, n):
    return rng.standard_normal(n) * np.exp(rng.uniform(-12, 6, n))


def test_round_bf16_matches_torch_conversion_on_float32_inputs():
    rng = np.random.default_rng(0)
    x = _scale_mix(rng, 20000).astype(np.float32)
    # exact ties between two bfloat16 neighbours, even and odd kept bit
    u = (rng.integers(0x3F000000, 0x42000000, 4000, dtype=np.uint32) & 0xFFFF0000) | 0x8000
    x = np.concatenate([x, u.view(np.float32), -u.view(np.float32)])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(O.round_bf16(x), ref)


def test_round_bf16_is_nearest_with_eight_significant_bits():
    rng = np.random.default_rng(1)
    x = _scale_mix(rng, 5000)
    r = O.round_bf16(x)
    m, e = np.frexp(r)
    assert np.array_equal(np.ldexp(m, 8), np.round(np.ldexp(m, 8)))  # 8 significant bits
    _, ex = np.frexp(x)
    ulp = np.ldexp(1.0, ex - 8)
    assert np.all(np.abs(x - r) <= ulp / 2)
    assert np.all(np.abs(r) <= np.abs(x) * (1 + 2.0**-8))


def test_round_fp16_matches_torch_conversion():
    rng = np.random.default_rng(2)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-18, 8, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(O.round_fp16(x), ref)


def test_split_represents_value_to_sixteen_bits():
    rng = np.random.default_rng(3)
    x = _scale_mix(rng, 5000)
    hi = O.round_bf16(x)
    lo = O.round_bf16(x - hi)
    assert np.all(np.abs(lo) <= 2.0**-8 * np.abs(x) * (1 + 2.0**-7))
    assert np.all(np.abs(x - hi - lo) <= 2.0**-16 * np.abs(x))


def test_half_spectrum_operand_is_hermitian_with_real_ends():
    rng = np.random.default_rng(4)
    c = rng.standard_normal((3, 5, 32)) + 1j * rng.standard_normal((3, 5, 32))
    h = O.half_spectrum_operand(c)
    assert np.all(h[..., 0].imag == 0) and np.all(h[..., 16].imag == 0)
    assert np.array_equal(h[..., 1:16], c[..., 1:16])
    assert np.array_equal(h[..., 17:], np.conj(h[..., 1:16][..., ::-1]))


def _small():
    wl = make_workload(N=32, R=16, Q=32, N_B=5, N_A=6, snr=0.2, T_side=2, seed=21)
    g = wl.grid
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), 8)
    a = O.compress(O.translate(wl.images, g.k, wl.deltas), U, g.w)
    b = O.compress(wl.templates, U, g.w)
    return a, b


def test_forms_reduce_to_the_exact_score_on_representable_operands():
    a, b = _small()
    rb = lambda z: O.round_bf16(z.real) + 1j * O.round_bf16(z.imag)
    a16, b16 = rb(O.half_spectrum_operand(a)), rb(O.half_spectrum_operand(b))
    X = O.scores_compressed(a16, b16).real
    for form in ("bf16", "bf16x3", "fp64"):
        Xf = O.scores_compressed_form(a16, b16, form)
        assert np.allclose(Xf, X, rtol=0, atol=1e-13 * np.abs(X).max()), form
    rh = lambda z: O.round_fp16(z.real) + 1j * O.round_fp16(z.imag)
    ah, bh = rh(O.half_spectrum_operand(a)), rh(O.half_spectrum_operand(b))
    Xh = O.scores_compressed(ah, bh).real
    assert np.allclose(O.scores_compressed_form(ah, bh, "fp16"), Xh, rtol=0, atol=1e-13 * np.abs(Xh).max())


def test_fp64_form_of_real_image_rings_is_the_plain_score():
    a, b = _small()
    X = O.scores_compressed(a, b).real
    assert np.allclose(O.scores_compressed_form(a, b, "fp64"), X, rtol=0, atol=1e-12 * np.abs(X).max())


def test_form_errors_follow_the_rounding_bounds():
    """bf16x3 keeps about 16 significand bits: relative error far below the
    single-pass forms, and dropping any one of its three terms is visible."""
    a, b = _small()
    X = O.scores_compressed(a, b).real
    nrm = np.linalg.norm(X)
    err = {f: np.linalg.norm(O.scores_compressed_form(a, b, f) - X) / nrm for f in ("bf16", "fp16", "bf16x3")}
    assert 1e-4 < err["bf16"] < 1e-2
    assert 1e-5 < err["fp16"] < 2e-3
    assert err["bf16x3"] < 1e-5
    assert err["bf16x3"] < err["fp16"] / 10
    terms = O.operand_terms(a, b, "bf16x3")
    for drop in range(3):
        kept = [t for i, t in enumerate(terms) if i != drop]
        Xhat = sum(2 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(A), B) for A, B in kept)
        e = np.linalg.norm(np.fft.fft(Xhat, axis=-1).real - X) / nrm
        assert e > 10 * err["bf16x3"], drop


def test_every_operand_is_a_value_of_its_format():
    """The tensor cores take bf16 (or fp16) values only: every operand of the
    single-pass forms, and the hi and lo parts of the split form, is unchanged by
    rounding to that format (checked against torch's conversion)."""
    rng = np.random.default_rng(11)
    a = (rng.standard_normal((2, 1, 3, 16)) + 1j * rng.standard_normal((2, 1, 3, 16))) * 3.7
    b = (rng.standard_normal((2, 3, 16)) + 1j * rng.standard_normal((2, 3, 16))) * 0.01

    def representable(z, dtype):
        for part in (z.real, z.imag):
            t = torch.from_numpy(np.ascontiguousarray(part)).to(torch.float32)
            if not np.array_equal(t.to(dtype).to(torch.float64).numpy(), part):
                return False
        return True

    for form, dtype in (("bf16", torch.bfloat16), ("fp16", torch.float16), ("bf16x3", torch.bfloat16)):
        for A, B in O.operand_terms(a, b, form):
            assert representable(A, dtype) and representable(B, dtype), form


def test_pow2_row_scale_puts_each_row_maximum_in_one_binade():
    """fp16x3 scaling: per row (leading indices) a power of two 2^e with the
    row's largest component in [2^13, 2^14) after scaling, undone exactly by
    the returned factor; a zero row keeps factor 1."""
    rng = np.random.default_rng(12)
    z = (rng.standard_normal((4, 3, 5, 16)) + 1j * rng.standard_normal((4, 3, 5, 16)))
    z *= np.exp(rng.uniform(-30, 30, (4, 3, 1, 1)))
    z[1, 2] = 0
    zs, f = O.pow2_row_scale(z)
    m = np.maximum(np.abs(zs.real), np.abs(zs.imag)).max(axis=(-2, -1))
    live = np.ones((4, 3), bool)
    live[1, 2] = False
    assert np.all((m[live] >= 2.0**13) & (m[live] < 2.0**14))
    assert f[1, 2, 0, 0] == 1.0 and np.all(zs[1, 2] == 0)
    mant, _ = np.frexp(f)
    assert np.all(mant == 0.5)  # powers of two
    assert np.array_equal(zs * f, z)


def test_fp16x3_parts_are_half_values_keeping_22_bits():
    """The hi and lo parts of the scaled split are IEEE half values (torch's
    conversion leaves them unchanged) and represent the scaled component to
    2^-22 relative (or the half subnormal spacing 2^-24 / 2 absolute)."""
    a, b = _small()
    for z, terms_side in ((O.half_spectrum_operand(a), 0), (O.half_spectrum_operand(b), 1)):
        zs, f = O.pow2_row_scale(z)
        terms = O.operand_terms(a, b, "fp16x3")
        hi = terms[0][terms_side] / f
        lo = (terms[2][0] / f) if terms_side == 0 else (terms[1][1] / f)
        for part in (hi.real, hi.imag, lo.real, lo.imag):
            t = torch.from_numpy(np.ascontiguousarray(part)).to(torch.float32)
            assert np.array_equal(t.to(torch.float16).to(torch.float64).numpy(), part)
        for x, h, l in ((zs.real, hi.real, lo.real), (zs.imag, hi.imag, lo.imag)):
            assert np.all(np.abs(x - h - l) <= np.maximum(2.0**-22 * np.abs(x), 2.0**-25))


def test_fp16x3_is_invariant_under_power_of_two_scaling():
    """Scaling the images by 2^k scales the fp16x3 score by exactly 2^k, far
    outside half precision's range (the per-row scaling absorbs it)."""
    a, b = _small()
    X0 = O.scores_compressed_form(a, b, "fp16x3")
    for k in (-60, -17, 23, 50):
        assert np.array_equal(O.scores_compressed_form(a * 2.0**k, b, "fp16x3"), 2.0**k * X0), k
        assert np.array_equal(O.scores_compressed_form(a, b * 2.0**k, "fp16x3"), 2.0**k * X0), k


def test_fp16x3_error_is_far_below_bf16x3_and_needs_every_term():
    a, b = _small()
    X = O.scores_compressed(a, b).real
    nrm = np.linalg.norm(X)
    e3 = np.linalg.norm(O.scores_compressed_form(a, b, "fp16x3") - X) / nrm
    eb = np.linalg.norm(O.scores_compressed_form(a, b, "bf16x3") - X) / nrm
    assert e3 < 2e-7 and e3 < eb / 20
    terms = O.operand_terms(a, b, "fp16x3")
    for drop in range(3):
        kept = [t for i, t in enumerate(terms) if i != drop]
        Xhat = sum(2 * math.pi * np.einsum("nthq,jhq->ntjq", np.conj(A), B) for A, B in kept)
        assert np.linalg.norm(np.fft.fft(Xhat, axis=-1).real - X) / nrm > 10 * e3, drop


def test_fp16x3_is_exact_on_operands_representable_after_scaling():
    """Rows whose scaled components are already half values pass through the
    split unchanged (lo = 0): the score is the exact one."""
    a, b = _small()
    A, B = O.half_spectrum_operand(a), O.half_spectrum_operand(b)
    rh = lambda z: O.round_fp16(z.real) + 1j * O.round_fp16(z.imag)
    (As, fa), (Bs, fb) = O.pow2_row_scale(A), O.pow2_row_scale(B)
    A16, B16 = rh(As) * fa, rh(Bs) * fb
    X = O.scores_compressed(A16, B16).real
    assert np.allclose(O.scores_compressed_form(A16, B16, "fp16x3"), X, rtol=0, atol=1e-13 * np.abs(X).max())
