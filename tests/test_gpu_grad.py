"""Differentiation path on the GPU (through the C ABI) against the FP64 oracle:
log-sum-exp rows, the adjoint of the fused scoring (gradient with respect to
the compressed rings), the adjoint of the compression, the end-to-end
torch.autograd.Function, central finite differences, and the 4096-image x
256-template differentiation workload on sampled outputs.

Gradient tolerance: P = s gL exp(s X - L) turns an absolute error e in X into
a relative error s e in P; with the FP32 X error below 1e-6 of the landscape
scale (|X| ~ 10) this is a few 1e-6, so gradients are compared normwise at
GTOL = 5e-5 of their largest entry."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from synthetic import make_workload  # noqa: E402
from tests.gpu_common import pack_slots  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"
GTOL = 5e-5


def unpack_full(c):
    """packed slots [..., H, M, 2] -> full spectrum [..., H, Q] with the pairing
    c(Q - q) = (-1)^q conj(c(q))."""
    M = c.shape[-2]
    Q = 2 * M
    z = c[..., 0] + 1j * c[..., 1]
    out = np.zeros(c.shape[:-2] + (Q,), dtype=np.complex128)
    out[..., 1:M] = z[..., 1:]
    out[..., 0] = c[..., 0, 0]
    out[..., M] = c[..., 0, 1]
    q = np.arange(M + 1, Q)
    out[..., q] = ((-1.0) ** q) * np.conj(out[..., Q - q])
    return out


def _setup(Q, R, H, T_side, N_A, N_B, seed):
    wl = make_workload(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, snr=0.05, T_side=T_side, seed=seed)
    A = wl.images.astype(np.complex64)
    B = wl.templates.astype(np.complex64)
    U, _ = O.principal_vectors(O.radial_kernel(B.astype(np.complex128), wl.grid.w), H)
    return wl, A, B, U


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_lse_rows_matches_logsumexp():
    from scipy.special import logsumexp

    rng = np.random.default_rng(0)
    x = (5 * rng.standard_normal((37, 301))).astype(np.float32)
    L = P.lse_rows(torch.from_numpy(x).to(DEV)).cpu().numpy()
    assert np.max(np.abs(L - logsumexp(x.astype(np.float64), axis=1))) < 1e-5 * np.max(np.abs(L))


GRAD_CASES = [
    # (Q, R, H, T_side, N_A, N_B, inv_sigma2)
    (256, 64, 12, 3, 5, 7, 1.0),   # differentiation geometry, ragged
    (128, 32, 8, 1, 9, 5, 1.0),
    (128, 32, 32, 1, 4, 3, 0.5),   # H = 32
    (512, 48, 16, 2, 3, 4, 1.0),   # Q = 512
    (256, 40, 20, 1, 6, 5, 2.0),   # H padded to 24
]


@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B,s", GRAD_CASES)
def test_lse_backward_matches_oracle(Q, R, H, T_side, N_A, N_B, s):
    wl, A, B, U = _setup(Q, R, H, T_side, N_A, N_B, seed=Q + H + N_A)
    g = wl.grid
    T = wl.deltas.shape[0]
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas if T > 1 else None)
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV))
    _, _, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=s, want_lse=True)
    L = P.lse_rows(lse)
    rng = np.random.default_rng(1)
    gL = (0.5 + rng.random(N_A)).astype(np.float32)
    gA, gB = P.lse_backward(cA, N_A, T, cB, N_B, H, Q, s, L, torch.from_numpy(gL).to(DEV))
    P.status()
    a_c = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b_c = O.compress(B.astype(np.complex128), U, g.w)
    loss, Ln, G_ac, G_bc = O.lse_grad_compressed(a_c, b_c, s, gL.astype(np.float64))
    assert np.max(np.abs(L.cpu().numpy() - Ln)) < 1e-5 * np.max(np.abs(Ln))
    ref_a = pack_slots(G_ac).reshape(N_A * T, H, Q // 2, 2)
    ref_b = pack_slots(G_bc).reshape(N_B, H, Q // 2, 2)
    assert _rel(gA.cpu().numpy(), ref_a) < GTOL
    assert _rel(gB.cpu().numpy(), ref_b) < GTOL


@pytest.mark.parametrize("Q,R,H,T_side", [(256, 64, 12, 3), (128, 32, 8, 1), (512, 20, 5, 2), (1024, 16, 16, 1)])
def test_compress_backward_matches_oracle_adjoint(Q, R, H, T_side):
    wl, A, B, U = _setup(Q, R, H, T_side, 3, 2, seed=7)
    g = wl.grid
    T = wl.deltas.shape[0]
    rng = np.random.default_rng(2)
    gC = rng.standard_normal((3 * T, H, Q // 2, 2)).astype(np.float32)
    out = P.compress_backward(g.k, g.w, torch.from_numpy(U).to(DEV), torch.from_numpy(gC).to(DEV), 3, R, Q,
                              deltas=wl.deltas if T > 1 else None).cpu().numpy()
    full = unpack_full(gC.astype(np.float64)).reshape(3, T, H, Q)
    ref = O.compress_adjoint(full, U, g.w, g.k, wl.deltas)
    assert _rel(out, ref) < 1e-5


def test_lse_align_autograd_matches_oracle_gradient():
    wl, A, B, U = _setup(256, 64, 12, 3, 6, 5, seed=31)
    g = wl.grid
    s = 1.0
    At = torch.from_numpy(A).to(DEV).requires_grad_(True)
    Bt = torch.from_numpy(B).to(DEV).requires_grad_(True)
    L = P.lse_align(At, Bt, torch.from_numpy(U).to(DEV), g.k, g.w, wl.deltas, s)
    L.sum().backward()
    P.status()
    loss, GA, GB = O.lse_loss_grad(A.astype(np.complex128), B.astype(np.complex128), g.k, g.w, wl.deltas, U, s)
    assert abs(float(L.detach().sum()) - loss) < 1e-5 * abs(loss)
    assert _rel(At.grad.cpu().numpy(), GA) < GTOL
    assert _rel(Bt.grad.cpu().numpy(), GB) < GTOL


def test_lse_align_gradient_finite_differences_fp32():
    """Central differences of the GPU loss along Hermitian-paired random
    directions (the inputs are transforms of real images)."""
    wl, A, B, U = _setup(128, 32, 8, 3, 4, 3, seed=41)
    g = wl.grid
    Ut = torch.from_numpy(U).to(DEV)
    At = torch.from_numpy(A).to(DEV).requires_grad_(True)
    Bt = torch.from_numpy(B).to(DEV).requires_grad_(True)
    L = P.lse_align(At, Bt, Ut, g.k, g.w, wl.deltas, 1.0).sum()
    L.backward()
    GA, GB = At.grad.cpu().numpy().astype(np.complex128), Bt.grad.cpu().numpy().astype(np.complex128)
    rng = np.random.default_rng(5)
    M = g.Q // 2

    def loss(a, b):
        with torch.no_grad():
            return float(P.lse_align(torch.from_numpy(a).to(DEV), torch.from_numpy(b).to(DEV), Ut, g.k, g.w,
                                     wl.deltas, 1.0).double().sum())

    for which, base, G in (("images", A, GA), ("templates", B, GB)):
        for _ in range(3):
            v = rng.standard_normal(base.shape[:-1] + (M,)) + 1j * rng.standard_normal(base.shape[:-1] + (M,))
            v = np.concatenate([v, np.conj(v)], axis=-1)
            v *= np.linalg.norm(base) / np.linalg.norm(v) * 1e-2
            a_p, a_m, b_p, b_m = A, A, B, B
            if which == "images":
                a_p, a_m = (A + v).astype(np.complex64), (A - v).astype(np.complex64)
            else:
                b_p, b_m = (B + v).astype(np.complex64), (B - v).astype(np.complex64)
            fd = (loss(a_p, b_p) - loss(a_m, b_m)) / 2.0
            an = float(np.sum(np.real(np.conj(G) * v)))
            assert abs(fd - an) <= 2e-2 * abs(an) + 1e-4, (which, fd, an)


@pytest.mark.parametrize("Q,R,H,T_side", [(256, 64, 12, 3), (512, 48, 16, 2)])
def test_lse_backward_accumulated_over_image_batches(Q, R, H, T_side):
    """The images streamed through in three batches, each batch's template
    gradient added into one gB (rsvd_lse_backward_accumulate): against the
    oracle gradient of the whole set; the image gradients of each batch
    against the oracle rows of that batch."""
    N_A, N_B = 11, 6
    wl, A, B, U = _setup(Q, R, H, T_side, N_A, N_B, seed=Q + 3 * H)
    g = wl.grid
    T = wl.deltas.shape[0]
    Ut = torch.from_numpy(U).to(DEV)
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV))
    gB = torch.zeros_like(cB)
    gAs = []
    for n0, n1 in ((0, 4), (4, 9), (9, 11)):
        n = n1 - n0
        cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A[n0:n1]).to(DEV), deltas=wl.deltas)
        _, _, lse = P.align_best(cA, n, T, cB, N_B, H, Q, want_lse=True)
        L = P.lse_rows(lse)
        gL = torch.ones(n, dtype=torch.float32, device=DEV)
        gA, _ = P.lse_backward(cA, n, T, cB, N_B, H, Q, 1.0, L, gL, gB=gB, accumulate=True)
        gAs.append(gA.cpu().numpy())
    P.status()
    a_c = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b_c = O.compress(B.astype(np.complex128), U, g.w)
    _, _, G_ac, G_bc = O.lse_grad_compressed(a_c, b_c, 1.0)
    assert _rel(gB.cpu().numpy(), pack_slots(G_bc).reshape(N_B, H, Q // 2, 2)) < GTOL
    ref_a = pack_slots(G_ac).reshape(N_A * T, H, Q // 2, 2)
    assert _rel(np.concatenate(gAs), ref_a) < GTOL


def test_differentiation_workload_sampled_parity():
    """4096 images x 256 templates, 128 px, 64 rings, Q = 256, 3x3 translations,
    H = 12, sigma^2 = 1: forward and backward on the GPU; the gradient of 8
    sampled images is checked against the oracle evaluated on those images and
    all templates, and the template gradient through the exact identity
    d/de L((1+e) templates) = d/de L((1+e) images) (both equal
    sum over pairs of dL/dX * X), evaluated on the packed gradients."""
    from synthetic import CONFIGS, make_workload_torch

    cfg = CONFIGS["gradient"]
    grid, deltas, tmpl, imgs, _ = make_workload_torch(**cfg, seed=3, device=DEV)
    H, Q = cfg["H"], cfg["Q"]
    N_A, N_B = cfg["N_A"], cfg["N_B"]
    U, _ = P.build_radial_svd(grid.w, tmpl, H)
    cA = P.compress(grid.k, grid.w, U, imgs, deltas=deltas)
    cB = P.compress(grid.k, grid.w, U, tmpl)
    T = deltas.shape[0]
    _, _, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=True)
    L = P.lse_rows(lse)
    gL = torch.ones(N_A, dtype=torch.float32, device=DEV)
    gA, gB = P.lse_backward(cA, N_A, T, cB, N_B, H, Q, 1.0, L, gL)
    P.status()

    def packed_dot(G, x):  # sum of dL/dtheta * theta over the packed real parameters
        G = G.double()
        x = x.double()
        d0 = (G[..., 0, :] * x[..., 0, :]).sum()
        d1 = (G[..., 1:, :] * x[..., 1:, :]).sum()
        return float(d0 + 2 * d1)

    lhs, rhs = packed_dot(gB, cB), packed_dot(gA, cA)
    assert abs(lhs - rhs) < 1e-4 * abs(rhs)

    rng = np.random.default_rng(4)
    ns = np.sort(rng.choice(N_A, 8, replace=False))
    idx = torch.from_numpy(ns).to(DEV)
    A = imgs[idx].cpu().numpy().astype(np.complex128)
    B = tmpl.cpu().numpy().astype(np.complex128)
    Un = U.cpu().numpy()
    a_c = O.compress(O.translate(A, grid.k, deltas), Un, grid.w)
    b_c = O.compress(B, Un, grid.w)
    _, Ln, G_ac, _ = O.lse_grad_compressed(a_c, b_c, 1.0)
    assert np.max(np.abs(L[idx].cpu().numpy() - Ln)) < 1e-5 * np.max(np.abs(Ln))
    got = gA.view(N_A, T, H, Q // 2, 2)[idx].cpu().numpy()
    assert _rel(got, pack_slots(G_ac)) < GTOL


def test_differentiation_workload_template_gradient_elementwise():
    """Differentiation workload at full size (4096 images x 256 templates,
    Q = 256, 3x3 translations, H = 12, sigma^2 = 1): the gradient of 4 sampled
    templates, every element, against the FP64 oracle summed over all 4096
    images (chunks of 64 images on spawned host processes)."""
    import multiprocessing as mp
    import os

    from synthetic import CONFIGS, make_workload_torch
    from tests.gpu_common import oracle_template_grad_chunk

    cfg = CONFIGS["gradient"]
    grid, deltas, tmpl, imgs, _ = make_workload_torch(**cfg, seed=5, device=DEV)
    H, Q = cfg["H"], cfg["Q"]
    N_A, N_B = cfg["N_A"], cfg["N_B"]
    U, _ = P.build_radial_svd(grid.w, tmpl, H)
    cA = P.compress(grid.k, grid.w, U, imgs, deltas=deltas)
    cB = P.compress(grid.k, grid.w, U, tmpl)
    T = deltas.shape[0]
    _, _, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=True)
    L = P.lse_rows(lse)
    gL = torch.ones(N_A, dtype=torch.float32, device=DEV)
    _, gB = P.lse_backward(cA, N_A, T, cB, N_B, H, Q, 1.0, L, gL)
    P.status()

    rng = np.random.default_rng(6)
    jsel = np.sort(rng.choice(N_B, 4, replace=False))
    Un = U.cpu().numpy()
    B = tmpl.cpu().numpy().astype(np.complex128)
    b_c = O.compress(B, Un, grid.w)
    A_all = imgs.cpu().numpy()
    jobs = []
    for n0 in range(0, N_A, 64):
        A = A_all[n0:n0 + 64].astype(np.complex128)
        jobs.append((O.compress(O.translate(A, grid.k, deltas), Un, grid.w), b_c, 1.0, jsel))
    n = min(len(os.sched_getaffinity(0)), 16)
    with mp.get_context("spawn").Pool(n) as pool:
        parts = pool.map(oracle_template_grad_chunk, jobs)
    G_ref = np.sum(parts, axis=0)  # [4, H, Q] full spectrum
    got = gB.view(N_B, H, Q // 2, 2)[torch.from_numpy(jsel).to(DEV)].cpu().numpy()
    assert _rel(got, pack_slots(G_ref)) < GTOL
