"""Sanity of the seeded input generator (no method arithmetic involved)."""

import math

import numpy as np

from synthetic import CONFIGS, make_workload, polar_grid, polar_norm2, translation_grid


def test_grid_constants():
    g = polar_grid(128, 64, 256)
    assert abs(g.K - 0.5 * math.pi * 128) < 1e-12
    assert abs(g.dk - math.pi) < 1e-12  # R = N/2 gives the unit-bandlimit spacing
    assert abs(g.k[-1] - g.K) < 1e-12 and abs(g.k[0] - g.dk) < 1e-12
    assert abs(g.w[-1] - 0.5 * g.k[-1] * g.dk) < 1e-12
    # trapezoid integrates k dk exactly over [0, K] for g = 1
    assert abs(g.w.sum() - 0.5 * g.K ** 2) < 1e-9 * g.K ** 2


def test_translation_grid_layout():
    d = translation_grid(128, 3)
    assert d.shape == (9, 2)
    px = 2.0 / 128
    assert np.allclose(d[0], (-px, -px)) and np.allclose(d[4], (0, 0)) and np.allclose(d[5], (px, 0))


def test_workload_is_seeded_hermitian_and_at_requested_snr():
    a = make_workload(N=64, R=32, Q=128, N_B=8, N_A=64, snr=0.1, seed=0)
    b = make_workload(N=64, R=32, Q=128, N_B=8, N_A=64, snr=0.1, seed=0)
    assert np.array_equal(a.images, b.images) and np.array_equal(a.templates, b.templates)
    h = a.grid.Q // 2
    for F in (a.images, a.templates):
        assert np.max(np.abs(F[..., h:] - np.conj(F[..., :h]))) < 1e-12 * np.max(np.abs(F))
    clean = make_workload(N=64, R=32, Q=128, N_B=8, N_A=64, snr=None, seed=0)
    sig = polar_norm2(a.grid, clean.images)
    noise = polar_norm2(a.grid, a.images - clean.images)
    ratio = np.mean(sig) / np.mean(noise)
    assert 0.08 < ratio < 0.125


def test_configs_have_expected_shapes():
    c = CONFIGS["throughput"]
    assert (c["N"], c["R"], c["Q"], c["N_B"], c["N_A"], c["T_side"], c["H"]) == (128, 64, 256, 1024, 8192, 3, 12)
