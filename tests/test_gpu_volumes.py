"""Volume alignment (section 4) through the C ABI against the FP64 oracle."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import volumes_ref as V  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402
from synthetic.volumes import make_volume_workload  # noqa: E402

DEV = "cuda:0"
RTOL = 1e-5


def _wl(L=8, R=8, N_B=3, N_A=5, n_beta=9, Mp=32, snr=0.5, seed=0):
    wl = make_volume_workload(N=2 * R, R=R, L=L, N_B=N_B, N_A=N_A, snr=snr, n_beta=n_beta, Mp=Mp, seed=seed)
    A = wl.volumes.astype(np.complex64)
    B = wl.targets.astype(np.complex64)
    return wl, A, B


def _eig_check(Ug, eg, Ur, lam, H):
    assert np.max(np.abs(eg - lam)) <= 1e-9 * max(abs(lam[0]), 1e-300)
    ext = np.r_[np.inf, lam, -np.inf]
    gaps = np.minimum(ext[0:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
    for h in range(H):
        if gaps[h] > 1e-6 * lam[0]:
            assert np.max(np.abs(Ug[:, h] - Ur[:, h])) < 1e-6, h


@pytest.mark.parametrize("L,R,N_B,HC,HD", [(8, 8, 3, 5, 6), (16, 12, 2, 8, 8), (24, 16, 1, 8, 8)])
def test_volume_svd_matches_oracle(L, R, N_B, HC, HD):
    wl, A, B = _wl(L=L, R=R, N_B=N_B, N_A=1, n_beta=2, Mp=64, seed=L)
    g = wl.grid
    U, eU, Vd, eV = P.build_volume_svd(g.w, torch.from_numpy(B).to(DEV), HC, HD)
    P.status()
    Bd = B.astype(np.complex128)
    Ur, lu = V.volume_principal(V.volume_radial_kernel(Bd, g.w), HC)
    Vr, lv = V.volume_principal(V.volume_degree_kernel(Bd, g.w), HD)
    _eig_check(U.cpu().numpy(), eU.cpu().numpy(), Ur, lu, HC)
    _eig_check(Vd.cpu().numpy(), eV.cpu().numpy(), Vr, lv, HD)


def test_volume_tables_match_wigner_d():
    L, HD = 20, 6
    rng = np.random.default_rng(1)
    Vm = np.linalg.qr(rng.standard_normal((L + 1, L + 1)))[0][:, :HD]
    betas = np.array([0.0, 0.37, 1.1, np.pi / 2, 2.4, np.pi])
    T = P.volume_tables(torch.from_numpy(Vm).to(DEV), betas).cpu().numpy()
    P.status()
    M = 2 * L + 1
    assert T.shape == (len(betas), M, M, 8)
    assert np.all(T[..., HD:] == 0)
    for b, beta in enumerate(betas):
        ref = np.zeros((HD, M, M))
        for l in range(L + 1):
            s = slice(L - l, L + l + 1)
            ref[:, s, s] += Vm[l][:, None, None] * V.wigner_d(l, beta)[None]
        got = np.moveaxis(T[b, :, :, :HD], -1, 0)
        assert np.max(np.abs(got - ref)) <= 2e-6 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("HC", [3, 7, 13])
def test_compress_volume_matches_oracle(HC):
    wl, A, B = _wl(L=12, R=14, N_A=4, seed=3)
    g = wl.grid
    rng = np.random.default_rng(2)
    U = np.linalg.qr(rng.standard_normal((g.R, g.R)))[0][:, :HC]
    got = P.compress_volume(g.w, torch.from_numpy(U).to(DEV), torch.from_numpy(A).to(DEV)).cpu().numpy()
    P.status()
    ref = V.compress_volume(A.astype(np.complex128), U, g.w)
    L = g.L
    mask = np.abs(np.arange(-L, L + 1))[None, :] <= np.arange(L + 1)[:, None]
    assert np.max(np.abs(got - ref)[..., mask]) <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("L,R,HC,HD,n_beta,Mp,N_A,N_B", [(8, 8, 5, 6, 9, 32, 5, 3), (12, 10, 8, 8, 7, 32, 3, 2),
                                                          (24, 12, 8, 8, 5, 64, 2, 2), (7, 6, 6, 8, 6, 16, 4, 2),
                                                          (10, 8, 6, 6, 5, 64, 3, 2), (20, 10, 7, 5, 4, 64, 2, 1),
                                                          (28, 12, 6, 8, 4, 64, 2, 1)])
def test_align_volumes_matches_oracle(L, R, HC, HD, n_beta, Mp, N_A, N_B):
    wl, A, B = _wl(L=L, R=R, N_B=N_B, N_A=N_A, n_beta=n_beta, Mp=Mp, seed=L + Mp)
    g = wl.grid
    Bd, Ad = B.astype(np.complex128), A.astype(np.complex128)
    Ur, _ = V.volume_principal(V.volume_radial_kernel(Bd, g.w), HC)
    Vr, _ = V.volume_principal(V.volume_degree_kernel(Bd, g.w), HD)
    Ut, Vt = torch.from_numpy(Ur).to(DEV), torch.from_numpy(Vr).to(DEV)
    cA = P.compress_volume(g.w, Ut, torch.from_numpy(A).to(DEV))
    cB = P.compress_volume(g.w, Ut, torch.from_numpy(B).to(DEV))
    T = P.volume_tables(Vt, wl.betas)
    best, arg = P.align_volumes(cA, cB, Vt, T, Mp)
    P.status()
    X = V.volume_scores_compressed(V.compress_volume(Ad, Ur, g.w), V.compress_volume(Bd, Ur, g.w), Vr, wl.betas, Mp)
    rb, ra = V.volume_align_best(X)
    best, arg = best.cpu().numpy(), arg.cpu().numpy()
    flat = X.reshape(N_A, N_B, -1)
    scale = np.abs(flat).max(axis=-1)
    assert np.all(np.abs(best - rb) <= RTOL * scale)
    at = np.take_along_axis(flat, arg[..., None].astype(np.int64), axis=-1)[..., 0]
    assert np.all((arg == ra) | (at >= rb - RTOL * scale))


def test_full_rank_noiseless_volumes_recover_the_rotation():
    L, R, Mp, n_beta = 7, 6, 16, 9
    wl, A, B = _wl(L=L, R=R, N_B=2, N_A=6, n_beta=n_beta, Mp=Mp, snr=None, seed=11)
    g = wl.grid
    U, _, Vd, _ = P.build_volume_svd(g.w, torch.from_numpy(B).to(DEV), R, L + 1)
    cA = P.compress_volume(g.w, U, torch.from_numpy(A).to(DEV))
    cB = P.compress_volume(g.w, U, torch.from_numpy(B).to(DEV))
    best, arg = P.align_volumes(cA, cB, Vd, P.volume_tables(Vd, wl.betas), Mp)
    P.status()
    best, arg = best.cpu().numpy(), arg.cpu().numpy()
    truth = wl.truth_b * Mp * Mp + wl.truth_a * Mp + wl.truth_c
    assert np.array_equal(np.argmax(best, axis=1), wl.truth_j)
    for n in range(6):
        j = wl.truth_j[n]
        norm2 = float(np.einsum("rlm,r->", np.abs(B[j].astype(np.complex128)) ** 2, g.w))
        assert abs(best[n, j] - norm2) <= 1e-4 * norm2
        # beta = 0 and pi are degenerate (alpha and gamma combine); compare the score there
        if 0 < wl.truth_b[n] < n_beta - 1:
            assert arg[n, j] == truth[n]


def test_volume_limits_are_refused():
    L, HC, HD = 8, 4, 4
    M = 2 * L + 1
    c = torch.zeros((1, HC, L + 1, M), dtype=torch.complex64, device=DEV)
    Vd = torch.zeros((L + 1, HD), dtype=torch.float64, device=DEV)
    T = torch.zeros((2, M, M, 8), dtype=torch.float32, device=DEV)
    with pytest.raises(P.RSVDError):  # Mp below 2L + 1
        P.align_volumes(c, c, Vd, T, 16)
    with pytest.raises(P.RSVDError):  # Mp not a supported power of two
        P.align_volumes(c, c, Vd, T, 24)
    L2 = 31  # the compressed pair (2 x 8 x 32 x 63 complex values) exceeds shared memory
    c2 = torch.zeros((1, 8, L2 + 1, 2 * L2 + 1), dtype=torch.complex64, device=DEV)
    T2 = torch.zeros((1, 2 * L2 + 1, 2 * L2 + 1, 8), dtype=torch.float32, device=DEV)
    with pytest.raises(P.RSVDError):
        P.align_volumes(c2, c2, torch.zeros((L2 + 1, HD), dtype=torch.float64, device=DEV), T2, 64)
    with pytest.raises(P.RSVDError):  # H_D above the limit
        P.volume_tables(torch.zeros((L + 1, 9), dtype=torch.float64, device=DEV), [0.0, 1.0])
    P.status()


def test_volume_host_pipeline_equals_device_path():
    wl, A, B = _wl(L=12, R=10, N_B=3, N_A=23, n_beta=7, Mp=32, seed=21)
    g = wl.grid
    U, _, Vd, _ = P.build_volume_svd(g.w, torch.from_numpy(B).to(DEV), 8, 8)
    T = P.volume_tables(Vd, wl.betas)
    cA = P.compress_volume(g.w, U, torch.from_numpy(A).to(DEV))
    cB = P.compress_volume(g.w, U, torch.from_numpy(B).to(DEV))
    bd, ad = P.align_volumes(cA, cB, Vd, T, 32)
    bh, ah = P.align_volumes_host(g.w, U, Vd, T, 32, torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(),
                                  chunk=5)
    bhr, ahr = P.align_volumes_host(g.w, U, Vd, T, 32, torch.from_numpy(A).pin_memory(),
                                    torch.from_numpy(B).pin_memory(), chunk=5, real=True)
    brd, ard = P.align_volumes(cA, cB, Vd, T, 32, real=True)
    P.status()
    assert np.array_equal(bhr.numpy(), brd.cpu().numpy()) and np.array_equal(ahr.numpy(), ard.cpu().numpy())
    P.status()
    assert np.array_equal(bh.numpy(), bd.cpu().numpy())
    assert np.array_equal(ah.numpy(), ad.cpu().numpy())


@pytest.mark.parametrize("L,R,HC,HD,n_beta,Mp", [(8, 8, 5, 6, 9, 32), (24, 12, 8, 8, 5, 64), (7, 6, 6, 8, 6, 16)])
def test_real_volume_path_matches_general_path_and_oracle(L, R, HC, HD, n_beta, Mp):
    """Synthetic volumes are real (A_l^{-m} = (-1)^{l+m} conj A_l^m): the shortcut path
    agrees with the general one and with the oracle."""
    wl, A, B = _wl(L=L, R=R, N_B=2, N_A=4, n_beta=n_beta, Mp=Mp, seed=40 + L)
    g = wl.grid
    Bd, Ad = B.astype(np.complex128), A.astype(np.complex128)
    Ur, _ = V.volume_principal(V.volume_radial_kernel(Bd, g.w), HC)
    Vr, _ = V.volume_principal(V.volume_degree_kernel(Bd, g.w), HD)
    Ut, Vt = torch.from_numpy(Ur).to(DEV), torch.from_numpy(Vr).to(DEV)
    cA = P.compress_volume(g.w, Ut, torch.from_numpy(A).to(DEV))
    cB = P.compress_volume(g.w, Ut, torch.from_numpy(B).to(DEV))
    T = P.volume_tables(Vt, wl.betas)
    bg, ag = P.align_volumes(cA, cB, Vt, T, Mp)
    br, ar = P.align_volumes(cA, cB, Vt, T, Mp, real=True)
    P.status()
    X = V.volume_scores_compressed(V.compress_volume(Ad, Ur, g.w), V.compress_volume(Bd, Ur, g.w), Vr, wl.betas, Mp)
    rb, ra = V.volume_align_best(X)
    flat = X.reshape(4, 2, -1)
    scale = np.abs(flat).max(axis=-1)
    br, ar, bg = br.cpu().numpy(), ar.cpu().numpy(), bg.cpu().numpy()
    assert np.all(np.abs(br - bg) <= RTOL * scale)
    assert np.all(np.abs(br - rb) <= RTOL * scale)
    at = np.take_along_axis(flat, ar[..., None].astype(np.int64), axis=-1)[..., 0]
    assert np.all((ar == ra) | (at >= rb - RTOL * scale))
