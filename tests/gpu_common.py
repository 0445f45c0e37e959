"""Shared helpers for the GPU parity tests: seeded inputs, the FP64 oracle on
the same (complex64-rounded) inputs, and the comparison rules.

Tolerances (FP32 path against the FP64 oracle):
* scores X: |X_gpu - X_ref| <= RTOL * scale, scale = max |X_ref| over the
  landscape of that (image, template) pair, RTOL = 1e-5;
* best: same rule with the scale of the pair;
* arg: identical, or (several near-equal maxima) the oracle's own score at
  the GPU's argmax is within RTOL * scale of the oracle maximum;
* lse: |lse_gpu - lse_ref| <= RTOL * inv_sigma2 * scale (an FP32 error of
  eps in every X shifts the log-sum-exp by at most inv_sigma2 * eps).
"""

from __future__ import annotations

import math

import numpy as np

import oracle as O
from synthetic import make_workload

RTOL = 1e-5


def c64(x):
    return np.asarray(x, dtype=np.complex64)


def setup(N, R, Q, N_B, N_A, T_side=1, H=8, snr=0.1, seed=0):
    """Returns (wl, images64, templates64, U) with U from the oracle's kernel of
    the complex64-rounded templates."""
    wl = make_workload(N=N, R=R, Q=Q, N_B=N_B, N_A=N_A, snr=snr, T_side=T_side, seed=seed)
    A = c64(wl.images)
    B = c64(wl.templates)
    U, _ = O.principal_vectors(O.radial_kernel(B.astype(np.complex128), wl.grid.w), H)
    return wl, A, B, U


def oracle_scores(wl, A, B, U):
    g = wl.grid
    A_t = O.translate(A.astype(np.complex128), g.k, wl.deltas)
    a_c = O.compress(A_t, U, g.w)
    b_c = O.compress(B.astype(np.complex128), U, g.w)
    return O.scores_compressed(a_c, b_c).real, a_c, b_c


def pack_slots(c):
    """oracle compressed [..., H, Q] (full spectrum) -> packed slots [..., H, Q/2, 2]."""
    Q = c.shape[-1]
    M = Q // 2
    out = np.empty(c.shape[:-1] + (M, 2))
    out[..., 1:, 0] = c[..., 1:M].real
    out[..., 1:, 1] = c[..., 1:M].imag
    out[..., 0, 0] = c[..., 0].real
    out[..., 0, 1] = c[..., M].real
    return out


def check_best(X, best, arg, lse=None, inv_sigma2=1.0, exact_arg_mask=None):
    """X oracle [nA, T, nB, Q]; best/arg/lse GPU results (numpy)."""
    nA, T, nB, Q = X.shape
    flat = np.transpose(X, (0, 2, 1, 3)).reshape(nA, nB, T * Q)
    scale = np.max(np.abs(flat), axis=-1)
    rb, ra = O.align_best(X)
    err = np.abs(best - rb) / scale
    assert np.all(err <= RTOL), f"best max rel err {err.max():.3e}"
    ok = (arg == ra)
    at = np.take_along_axis(flat, np.clip(arg, 0, T * Q - 1)[..., None].astype(np.int64), axis=-1)[..., 0]
    near = (arg >= 0) & (arg < T * Q) & (at >= rb - RTOL * scale)
    assert np.all(ok | near), f"{np.sum(~(ok | near))} argmax mismatches beyond tolerance"
    if exact_arg_mask is not None:
        assert np.all(ok[exact_arg_mask]), "argmax differs on noiseless pairs"
    if lse is not None:
        rl = O.lse_pair_partials(X, inv_sigma2)
        lerr = np.abs(lse - rl) / (inv_sigma2 * scale)
        assert np.all(lerr <= RTOL), f"lse max err {lerr.max():.3e}"
    return float(err.max()), float(np.mean(ok))


def x_err(X_gpu, X_ref):
    nA, T, nB, Q = X_ref.shape
    scale = np.max(np.abs(X_ref), axis=-1, keepdims=True)
    return float(np.max(np.abs(X_gpu - X_ref) / scale))


def frob_rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def two_pi():
    return 2 * math.pi


def oracle_template_grad_chunk(job):
    """Oracle gradient of sum_n L_n with respect to the compressed templates
    `jsel`, summed over one chunk of images (each image's L_n spans every
    template, so the chunk's contribution is exact). Runs in a spawned worker."""
    a_c, b_c, inv_sigma2, jsel = job
    _, _, _, G_bc = O.lse_grad_compressed(a_c, b_c, inv_sigma2)
    return G_bc[jsel]
