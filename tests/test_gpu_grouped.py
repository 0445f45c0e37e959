"""Per-CTF principal vectors and grouped alignment (section 3.5) on the GPU
against the FP64 oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_common import check_best  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402
from synthetic import make_grouped_workload  # noqa: E402

DEV = "cuda:0"


@pytest.mark.parametrize("R,Q,N_B,G,H", [(32, 128, 12, 5, 8), (64, 256, 40, 17, 12), (20, 64, 7, 3, 20)])
def test_grouped_build_matches_oracle(R, Q, N_B, G, H):
    wl = make_grouped_workload(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=G, G=G, snr=None, seed=G + R)
    g = wl.grid
    S = wl.templates.astype(np.complex64)
    Ur, lam = O.grouped_principal_vectors(S.astype(np.complex128), g.w, wl.ctf, H)
    U, Ut, eig = P.build_radial_svd_grouped(g.w, torch.from_numpy(S).to(DEV), torch.from_numpy(wl.ctf).to(DEV), H)
    P.status()
    U, Ut, eig = U.cpu().numpy(), Ut.cpu().numpy(), eig.cpu().numpy()
    for gg in range(G):
        assert np.max(np.abs(eig[gg] - lam[gg])) <= 1e-10 * lam[gg][0]
        ext = np.r_[np.inf, lam[gg], -np.inf]
        gaps = np.minimum(ext[0:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
        for h in range(H):
            if gaps[h] > 1e-6 * lam[gg][0]:
                assert np.max(np.abs(U[gg][:, h] - Ur[gg][:, h])) < 1e-6, (gg, h)
        assert np.allclose(U[gg].T @ U[gg], np.eye(H), atol=1e-10)
        assert np.allclose(Ut[gg], wl.ctf[gg][:, None] * U[gg], rtol=0, atol=1e-15)


def test_grouped_alignment_matches_oracle():
    wl = make_grouped_workload(N=128, R=64, Q=256, N_B=9, N_A=23, G=4, snr=0.1, T_side=3, seed=6)
    g = wl.grid
    S = wl.templates.astype(np.complex64)
    A = wl.images.astype(np.complex64)
    H = 12
    U, Ut, _ = P.build_radial_svd_grouped(g.w, torch.from_numpy(S).to(DEV), torch.from_numpy(wl.ctf).to(DEV), H)
    best, arg = P.align_grouped(g.k, g.w, torch.from_numpy(A).to(DEV), wl.offsets, torch.from_numpy(S).to(DEV), U, Ut,
                                deltas=wl.deltas)
    P.status()
    Un = U.cpu().numpy()
    X = O.grouped_scores(A.astype(np.complex128), wl.offsets, S.astype(np.complex128), wl.ctf, Un, g.w, g.k,
                         wl.deltas)
    check_best(X, best.cpu().numpy(), arg.cpu().numpy())


def test_grouped_alignment_recovers_noiseless_truth():
    wl = make_grouped_workload(N=64, R=32, Q=128, N_B=6, N_A=15, G=3, snr=None, T_side=1, seed=9)
    g = wl.grid
    S = torch.from_numpy(wl.templates.astype(np.complex64)).to(DEV)
    U, Ut, _ = P.build_radial_svd_grouped(g.w, S, torch.from_numpy(wl.ctf).to(DEV), g.R)
    best, arg = P.align_grouped(g.k, g.w, torch.from_numpy(wl.images.astype(np.complex64)).to(DEV), wl.offsets, S, U,
                                Ut)
    P.status()
    best, arg = best.cpu().numpy(), arg.cpu().numpy()
    assert np.array_equal(np.argmax(best, axis=1), wl.truth_j)
    assert np.array_equal(arg[np.arange(15), wl.truth_j], wl.truth_m)


def test_grouped_alignment_is_the_same_on_any_number_of_streams():
    """Groups on 1 or 4 streams (round robin), including an empty and an odd-sized
    group, give bit-identical results: each group's kernels are independent."""
    wl = make_grouped_workload(N=128, R=64, Q=256, N_B=11, N_A=29, G=5, snr=0.1, T_side=3, seed=12)
    g = wl.grid
    S = torch.from_numpy(wl.templates.astype(np.complex64)).to(DEV)
    A = torch.from_numpy(wl.images.astype(np.complex64)).to(DEV)
    U, Ut, _ = P.build_radial_svd_grouped(g.w, S, torch.from_numpy(wl.ctf).to(DEV), 12)
    off = np.array([0, 7, 7, 18, 19, 29])  # group 1 empty, group 3 a single image
    b1, a1 = P.align_grouped(g.k, g.w, A, off, S, U, Ut, deltas=wl.deltas, n_streams=1)
    b4, a4 = P.align_grouped(g.k, g.w, A, off, S, U, Ut, deltas=wl.deltas, n_streams=4)
    P.status()
    assert torch.equal(b1, b4) and torch.equal(a1, a4)
    X = O.grouped_scores(wl.images.astype(np.complex64).astype(np.complex128), off,
                         wl.templates.astype(np.complex64).astype(np.complex128), wl.ctf, U.cpu().numpy(), g.w, g.k,
                         wl.deltas)
    check_best(X, b4.cpu().numpy(), a4.cpu().numpy())
