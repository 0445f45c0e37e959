"""Finer rotation grid (zero-padded X_hat, section 2.4), explicit pair lists and
principal-mode-marching (section 5) through the C ABI, against the FP64 oracle."""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_common import RTOL, check_best, setup  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"


def _compressed(wl, A, B, U):
    g = wl.grid
    T = wl.deltas.shape[0]
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas if T > 1 else None)
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV))
    a = O.compress(O.translate(A.astype(np.complex128), g.k, wl.deltas), U, g.w)
    b = O.compress(B.astype(np.complex128), U, g.w)
    return cA, cB, a, b, T


def _pair_err(Xg, Xr):
    nA, T, nB, _ = Xr.shape
    scale = np.max(np.abs(np.transpose(Xr, (0, 2, 1, 3)).reshape(nA, nB, -1)), axis=-1)
    return float((np.abs(Xg - Xr) / scale[:, None, :, None]).max())


@pytest.mark.parametrize("Q,R,H,T_side,Pf", [(128, 32, 8, 1, 2), (128, 32, 8, 2, 8), (256, 64, 12, 3, 4),
                                             (64, 16, 6, 1, 16), (32, 12, 5, 2, 4)])
def test_align_scores_fine_matches_oracle(Q, R, H, T_side, Pf):
    if Pf * Q > 1024 or Pf > 8:
        with pytest.raises(P.RSVDError):
            wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=3, N_A=2, T_side=T_side, H=H, seed=1)
            cA, cB, _, _, T = _compressed(wl, A, B, U)
            P.align_scores_fine(cA, 2, T, cB, 3, H, Q, Pf)
        return
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=5, N_A=7, T_side=T_side, H=H, seed=Q + Pf)
    cA, cB, a, b, T = _compressed(wl, A, B, U)
    X = P.align_scores_fine(cA, 7, T, cB, 5, H, Q, Pf).cpu().numpy().astype(np.float64)
    P.status()
    Xr = O.scores_fine(a, b, Pf)
    assert _pair_err(X, Xr) <= RTOL


def test_fine_grid_with_factor_one_is_the_plain_landscape():
    wl, A, B, U = setup(N=128, R=64, Q=256, N_B=4, N_A=3, T_side=2, H=12, seed=4)
    cA, cB, _, _, T = _compressed(wl, A, B, U)
    X1 = P.align_scores_fine(cA, 3, T, cB, 4, 12, 256, 1)
    X0 = P.align_scores(cA, 3, T, cB, 4, 12, 256)
    P.status()
    assert torch.equal(X1, X0)


@pytest.mark.parametrize("method", ["shifted", "pair"])
@pytest.mark.parametrize("Q,R,H,T_side,Pf", [(128, 32, 8, 2, 4), (256, 64, 12, 3, 2), (256, 64, 16, 1, 1)])
def test_align_best_fine_matches_oracle(Q, R, H, T_side, Pf, method):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=6, N_A=9, T_side=T_side, H=H, seed=7 * Pf)
    cA, cB, a, b, T = _compressed(wl, A, B, U)
    best, arg, lse = P.align_best_fine(cA, 9, T, cB, 6, H, Q, Pf, inv_sigma2=0.5, want_lse=True, method=method)
    P.status()
    check_best(O.scores_fine(a, b, Pf), best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 0.5)


@pytest.mark.parametrize("Q,R,H,T_side,Pf,N_A,N_B", [(512, 48, 16, 2, 2, 5, 4), (256, 64, 12, 1, 8, 4, 3),
                                                      (128, 32, 5, 3, 2, 37, 21)])
def test_shifted_fine_grid_beyond_the_pair_kernel(Q, R, H, T_side, Pf, N_A, N_B):
    """Shifted passes cover P Q > 1024 and run on the fused kernels (several tiles, ragged)."""
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=Q + Pf)
    cA, cB, a, b, T = _compressed(wl, A, B, U)
    best, arg, lse = P.align_best_fine(cA, N_A, T, cB, N_B, H, Q, Pf, want_lse=True)
    P.status()
    check_best(O.scores_fine(a, b, Pf), best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)


@pytest.mark.parametrize("method", ["shifted", "pair"])
def test_fine_grid_recovers_off_grid_rotations(method):
    """Noiseless images = templates rotated analytically by half-grid angles:
    at P = 2 the argmax lands on the odd fine angle 2 m0 + 1 for every image."""
    from synthetic.inputs import blobs_polar_ft, draw_blobs, polar_grid

    N, R, Q, Pf = 64, 32, 128, 2
    grid = polar_grid(N, R, Q)
    rng = np.random.default_rng(8)
    blobs = draw_blobs(rng, 6)
    m0 = rng.integers(0, Q, 6)
    B = blobs_polar_ft(grid, blobs).astype(np.complex64)
    A = blobs_polar_ft(grid, blobs, rotation=2 * math.pi * (m0 + 0.5) / Q).astype(np.complex64)
    U, _ = O.principal_vectors(O.radial_kernel(B.astype(np.complex128), grid.w), R)
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(grid.k, grid.w, Ut, torch.from_numpy(A).to(DEV))
    cB = P.compress(grid.k, grid.w, Ut, torch.from_numpy(B).to(DEV))
    best, arg, _ = P.align_best_fine(cA, 6, 1, cB, 6, R, Q, Pf, method=method)
    P.status()
    arg = arg.cpu().numpy()
    assert np.array_equal(np.diag(arg), 2 * m0 + 1)


def test_align_best_pairs_matches_full_alignment():
    wl, A, B, U = setup(N=128, R=64, Q=256, N_B=7, N_A=5, T_side=3, H=12, seed=9)
    cA, cB, a, b, T = _compressed(wl, A, B, U)
    rng = np.random.default_rng(0)
    pairs = np.stack([rng.integers(0, 5, 23), rng.integers(0, 7, 23)], axis=1).astype(np.int32)
    pt = torch.from_numpy(pairs).to(DEV)
    bp, ap, lp = P.align_best_pairs(cA, 5, T, cB, 7, 12, 256, pt, inv_sigma2=1.0, want_lse=True)
    bf, af, lf = P.align_best(cA, 5, T, cB, 7, 12, 256, want_lse=True, pairwise=True)
    P.status()
    n, j = pairs[:, 0], pairs[:, 1]
    assert np.array_equal(bp.cpu().numpy(), bf.cpu().numpy()[n, j])
    assert np.array_equal(ap.cpu().numpy(), af.cpu().numpy()[n, j])
    assert np.array_equal(lp.cpu().numpy(), lf.cpu().numpy()[n, j])
    Xr = O.scores_compressed(a, b).real
    # the oracle on the listed pairs
    rb, ra = O.align_best(Xr)
    scale = np.max(np.abs(Xr), axis=(1, 3))
    assert np.all(np.abs(bp.cpu().numpy() - rb[n, j]) <= RTOL * scale[n, j])


def test_align_best_pairs_flags_a_bad_pair():
    wl, A, B, U = setup(N=64, R=32, Q=128, N_B=3, N_A=2, H=8, seed=2)
    cA, cB, _, _, T = _compressed(wl, A, B, U)
    pt = torch.tensor([[0, 1], [2, 0], [1, 3]], dtype=torch.int32, device=DEV)
    best = torch.full((3,), 7.0, device=DEV)
    arg = torch.full((3,), -9, dtype=torch.int32, device=DEV)
    P.lib().rsvd_align_best_pairs(cA.data_ptr(), 2, T, cB.data_ptr(), 3, 8, 128, 1, 0, pt.data_ptr(), 3, 1.0,
                                  best.data_ptr(), arg.data_ptr(), None, torch.cuda.current_stream().cuda_stream)
    with pytest.raises(P.RSVDError):
        P.status()
    assert best[1].item() == 7.0 and best[2].item() == 7.0 and arg[1].item() == -9
    assert best[0].item() != 7.0


def test_select_pairs_takes_the_largest_scores_in_index_order():
    rng = np.random.default_rng(3)
    b = rng.standard_normal((37, 300)).astype(np.float32)
    b[5, 10:20] = 9.0  # ties: kept in increasing template index
    keep = 12
    pairs = P.select_pairs(torch.from_numpy(b).to(DEV), keep).cpu().numpy()
    P.status()
    for n in range(37):
        order = sorted(range(300), key=lambda j: (-b[n, j], j))[:keep]
        assert np.array_equal(pairs[n * keep:(n + 1) * keep, 0], np.full(keep, n))
        assert np.array_equal(pairs[n * keep:(n + 1) * keep, 1], order)


def test_principal_mode_marching_refines_to_the_high_rank_result():
    """Coarse pass at H = 4, keep 6 templates per image, refine at H = 16 on a
    2x finer grid: the refined scores equal the oracle's H = 16 fine landscape on
    the kept pairs, and every image whose true template survives the coarse pass
    gets the same argmax as the full H = 16 alignment."""
    wl, A, B, U = setup(N=64, R=32, Q=128, N_B=24, N_A=40, T_side=1, H=16, snr=0.1, seed=12)
    g = wl.grid
    Ut = torch.from_numpy(U).to(DEV)
    U4 = np.ascontiguousarray(U[:, :4])
    U4t = torch.from_numpy(U4).to(DEV)
    At, Bt = torch.from_numpy(A).to(DEV), torch.from_numpy(B).to(DEV)
    coarse = (P.compress(g.k, g.w, U4t, At), P.compress(g.k, g.w, U4t, Bt), 4)
    fine = (P.compress(g.k, g.w, Ut, At), P.compress(g.k, g.w, Ut, Bt), 16)
    pairs, b1, a1, _ = P.align_marching(coarse, fine, 40, 1, 24, 128, keep=6, P=2)
    P.status()
    pairs, b1, a1 = pairs.cpu().numpy(), b1.cpu().numpy(), a1.cpu().numpy()
    a = O.compress(A.astype(np.complex128)[:, None], U, g.w)
    b = O.compress(B.astype(np.complex128), U, g.w)
    Xf = O.scores_fine(a, b, 2)  # [40, 1, 24, 256]
    rb, ra = O.align_best(Xf)
    n, j = pairs[:, 0], pairs[:, 1]
    scale = np.max(np.abs(Xf), axis=(1, 3))
    assert np.all(np.abs(b1 - rb[n, j]) <= RTOL * scale[n, j])
    kept_truth = 0
    for img in range(40):
        rows = np.where(n == img)[0]
        if wl.truth_j[img] in j[rows]:
            kept_truth += 1
            r = rows[np.argmax(b1[rows])]
            jb = j[r]
            full_j = int(np.argmax(rb[img]))
            assert b1[r] >= rb[img, full_j] - RTOL * scale[img, full_j]
            if jb == full_j:
                assert a1[r] == ra[img, jb] or Xf[img, 0, jb, a1[r]] >= rb[img, jb] - RTOL * scale[img, jb]
    assert kept_truth >= 30
