"""Translation-aware principal vectors (section 5, eq.
Image_single_cost_with_translations) on the GPU against the FP64 oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402
from synthetic import make_workload, translation_grid  # noqa: E402

DEV = "cuda:0"


def _check(Ug, eg, Ur, lam, H):
    assert np.max(np.abs(eg - lam)) <= 1e-10 * lam[0]
    ext = np.r_[np.inf, lam, -np.inf]
    gaps = np.minimum(ext[0:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
    for h in range(H):
        if gaps[h] > 1e-6 * lam[0]:
            assert np.max(np.abs(Ug[:, h] - Ur[:, h])) < 1e-6, h
    assert np.allclose(Ug.T @ Ug, np.eye(H), atol=1e-10)


@pytest.mark.parametrize("R,Q,N_B,H,side,spacing,weighted", [(16, 32, 6, 6, 3, 1.0, False), (32, 64, 10, 8, 3, 2.0, True),
                                                             (24, 128, 7, 10, 5, 1.0, True)])
def test_translated_build_matches_oracle(R, Q, N_B, H, side, spacing, weighted):
    wl = make_workload(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=1, snr=None, seed=R + Q)
    g = wl.grid
    B = wl.templates.astype(np.complex64)
    deltas = translation_grid(2 * R, side, spacing)
    rng = np.random.default_rng(R)
    weights = rng.uniform(0.2, 1.0, deltas.shape[0]) if weighted else None
    K = O.radial_kernel_translated(B.astype(np.complex128), g.w, g.k, deltas, weights)
    Ur, lam = O.principal_vectors(K, H)
    Ug, eg = P.build_radial_svd_translated(g.k, g.w, torch.from_numpy(B).to(DEV), H, deltas, weights)
    P.status()
    _check(Ug.cpu().numpy(), eg.cpu().numpy(), Ur, lam, H)


def test_single_zero_translation_is_the_plain_build():
    wl = make_workload(N=128, R=64, Q=256, N_B=40, N_A=1, snr=None, seed=2)
    g = wl.grid
    Bt = torch.from_numpy(wl.templates.astype(np.complex64)).to(DEV)
    U0, e0 = P.build_radial_svd(g.w, Bt, 12)
    U1, e1 = P.build_radial_svd_translated(g.k, g.w, Bt, 12, np.zeros((1, 2)))
    P.status()
    e0, e1 = e0.cpu().numpy(), e1.cpu().numpy()
    assert np.max(np.abs(e0 - e1)) <= 1e-12 * e0[0]
    assert np.max(np.abs(U0.cpu().numpy() - U1.cpu().numpy())) < 1e-8


def test_translation_aware_vectors_capture_more_of_translated_scores():
    """The rank-H scores of translated images against templates are closer to the
    full-rank scores with the translation-aware vectors than with the plain ones
    (reported; the kernel averages the objective over the same translations)."""
    wl = make_workload(N=64, R=32, Q=128, N_B=32, N_A=32, snr=None, T_side=3, spacing_px=2.0, seed=4)
    g = wl.grid
    B = wl.templates.astype(np.complex64)
    Bt = torch.from_numpy(B).to(DEV)
    H = 6
    U0, _ = P.build_radial_svd(g.w, Bt, H)
    U1, _ = P.build_radial_svd_translated(g.k, g.w, Bt, H, wl.deltas)
    P.status()
    A = wl.images.astype(np.complex128)
    A_t = O.translate(A, g.k, wl.deltas)
    Bd = B.astype(np.complex128)
    Ufull, _ = O.principal_vectors(O.radial_kernel(Bd, g.w), g.R)
    X = O.scores_compressed(O.compress(A_t, Ufull, g.w), O.compress(Bd, Ufull, g.w)).real
    errs = []
    for U in (U0.cpu().numpy(), U1.cpu().numpy()):
        Xh = O.scores_compressed(O.compress(A_t, U, g.w), O.compress(Bd, U, g.w)).real
        errs.append(np.linalg.norm(Xh - X) / np.linalg.norm(X))
    print(f"\nrank-{H} relative error on X: plain U {errs[0]:.4e}, translation-aware U {errs[1]:.4e}")
    assert errs[1] < errs[0]
