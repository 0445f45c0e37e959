"""Pins for the oracle's hand-derived LSE-loss gradient: central finite
differences in FP64 and an independent route through torch CPU autograd."""

import math

import numpy as np
import pytest

import oracle as O
from synthetic import make_workload


def _setup(N, R, Q, N_B, N_A, T_side, H, seed):
    wl = make_workload(N=N, R=R, Q=Q, N_B=N_B, N_A=N_A, snr=0.05, T_side=T_side, seed=seed)
    g = wl.grid
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), H)
    return wl, g, U


def _loss(images, templates, g, deltas, U, s):
    A_t = O.translate(images, g.k, deltas)
    X = O.scores_compressed(O.compress(A_t, U, g.w), O.compress(templates, U, g.w)).real
    return O.lse_loss(X, s)[0]


@pytest.mark.parametrize("inv_sigma2", [1.0, 4.0])
def test_gradient_matches_central_differences(inv_sigma2):
    """16 images x 4 templates on the differentiation geometry (128 px, 64 rings,
    Q = 256, 3x3 translations, H = 12); central differences with step 1e-3 along
    random unit directions and on single coordinates."""
    wl, g, U = _setup(128, 64, 256, 4, 16, 3, 12, seed=21)
    s = inv_sigma2
    loss, GA, GB = O.lse_loss_grad(wl.images, wl.templates, g.k, g.w, wl.deltas, U, s)
    assert abs(loss - _loss(wl.images, wl.templates, g, wl.deltas, U, s)) < 1e-10 * abs(loss)
    rng = np.random.default_rng(3)
    h = 1e-3
    for which in ("images", "templates"):
        base = wl.images if which == "images" else wl.templates
        G = GA if which == "images" else GB
        for trial in range(3):
            v = rng.standard_normal(base.shape) + 1j * rng.standard_normal(base.shape)
            v /= np.linalg.norm(v)
            args_p = [wl.images, wl.templates]
            args_m = [wl.images, wl.templates]
            i = 0 if which == "images" else 1
            args_p[i] = base + h * v
            args_m[i] = base - h * v
            fd = (_loss(*args_p, g, wl.deltas, U, s) - _loss(*args_m, g, wl.deltas, U, s)) / (2 * h)
            an = np.sum(np.real(np.conj(G) * v))
            assert abs(fd - an) <= 1e-6 * max(abs(an), np.linalg.norm(G)), (which, trial, fd, an)
        # single coordinates: real and imaginary parts separately
        flat = np.argsort(-np.abs(G).ravel())[:2]
        for idx in flat:
            for unit in (1.0, 1j):
                e = np.zeros(base.size, dtype=np.complex128)
                e[idx] = unit
                e = e.reshape(base.shape)
                args_p = [wl.images, wl.templates]
                args_m = [wl.images, wl.templates]
                args_p[i] = base + h * e
                args_m[i] = base - h * e
                fd = (_loss(*args_p, g, wl.deltas, U, s) - _loss(*args_m, g, wl.deltas, U, s)) / (2 * h)
                an = np.real(np.conj(G.ravel()[idx]) * unit)
                assert abs(fd - an) <= 1e-6 * np.abs(G).max(), (which, idx, unit, fd, an)


def test_gradient_matches_torch_autograd():
    """The same loss written in torch FP64 ops, differentiated by autograd
    (torch's complex gradient is dL/dRe + i dL/dIm for a real loss)."""
    torch = pytest.importorskip("torch")
    wl, g, U = _setup(64, 32, 128, 5, 6, 3, 8, seed=22)
    s = 2.0
    loss, GA, GB = O.lse_loss_grad(wl.images, wl.templates, g.k, g.w, wl.deltas, U, s)
    A = torch.tensor(wl.images, requires_grad=True)
    B = torch.tensor(wl.templates, requires_grad=True)
    k = torch.tensor(g.k)
    psi = 2 * math.pi * torch.arange(g.Q, dtype=torch.float64) / g.Q
    d = torch.tensor(wl.deltas)
    ph = torch.exp(-1j * k[None, :, None] * (d[:, 0, None, None] * torch.cos(psi) + d[:, 1, None, None] * torch.sin(psi)))
    Wt = torch.tensor(U * np.sqrt(g.w)[:, None]).to(torch.complex128)
    a = torch.fft.fft(A[:, None] * ph[None], dim=-1) / g.Q
    b = torch.fft.fft(B, dim=-1) / g.Q
    ac = torch.einsum("rh,ntrq->nthq", Wt, a)
    bc = torch.einsum("rh,jrq->jhq", Wt, b)
    Xhat = 2 * math.pi * torch.einsum("nthq,jhq->ntjq", ac.conj(), bc)
    X = torch.fft.fft(Xhat, dim=-1).real
    L = torch.logsumexp(X.reshape(X.shape[0], -1) * s, dim=1).sum()
    L.backward()
    assert abs(L.item() - loss) < 1e-10 * abs(loss)
    np.testing.assert_allclose(A.grad.numpy(), GA, rtol=0, atol=1e-10 * np.abs(GA).max())
    np.testing.assert_allclose(B.grad.numpy(), GB, rtol=0, atol=1e-10 * np.abs(GB).max())
