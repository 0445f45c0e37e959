"""Parity of the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs. Sizes span several tiles with ragged tails; the last
test checks the full throughput workload on sampled outputs."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_common import RTOL, check_best, frob_rel, oracle_scores, pack_slots, setup, x_err  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"


def _gpu(wl, A, B, U):
    g = wl.grid
    At = torch.from_numpy(A).to(DEV)
    Bt = torch.from_numpy(B).to(DEV)
    Ut = torch.from_numpy(U).to(DEV)
    T = wl.deltas.shape[0]
    cA = P.compress(g.k, g.w, Ut, At, deltas=wl.deltas if T > 1 else None)
    cB = P.compress(g.k, g.w, Ut, Bt)
    return cA, cB, T


@pytest.mark.parametrize("Q,R,H,T_side", [(128, 32, 8, 1), (128, 32, 32, 1), (256, 64, 12, 3), (512, 48, 16, 2),
                                          (16, 6, 3, 1), (1024, 20, 5, 1),
                                          # tensor-core projection (rings beyond the shared-memory kernel):
                                          (256, 128, 16, 2), (512, 100, 11, 3), (512, 128, 16, 6)])
def test_compress_matches_oracle(Q, R, H, T_side):
    """Compressed rings against the oracle; R Q / 2 > 12,288 takes the
    tensor-core projection (3xTF32), including R not a multiple of 32, H < 16
    and 36 translations (two TMEM passes)."""
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=3, N_A=5, T_side=T_side, H=H, seed=Q + H)
    cA, cB, T = _gpu(wl, A, B, U)
    _, a_c, b_c = oracle_scores(wl, A, B, U)
    ref_a = pack_slots(a_c).reshape(5 * T, H, Q // 2, 2)
    ref_b = pack_slots(b_c).reshape(3, H, Q // 2, 2)
    got_a = cA.cpu().numpy()
    got_b = cB.cpu().numpy()
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        scale = np.max(np.abs(ref), axis=(1, 2, 3), keepdims=True)
        assert np.max(np.abs(got - ref) / scale) < RTOL
    P.status()


def test_compress_non_uniform_rings_tensor_core_projection():
    """Ring radii that are not equispaced through the tensor-core projection
    (per-ring phase evaluation)."""
    wl, A, B, U = setup(N=256, R=128, Q=512, N_B=2, N_A=2, T_side=3, H=16, seed=78)
    g = wl.grid
    rng = np.random.default_rng(4)
    k = np.sort(rng.uniform(1.0, g.K, size=g.R))
    w = rng.uniform(0.5, 2.0, size=g.R) * k
    At = torch.from_numpy(A).to(DEV)
    cA = P.compress(k, w, torch.from_numpy(U).to(DEV), At, deltas=wl.deltas).cpu().numpy()
    a_c = O.compress(O.translate(A.astype(np.complex128), k, wl.deltas), U, w)
    ref = pack_slots(a_c).reshape(2 * 9, 16, 256, 2)
    scale = np.max(np.abs(ref), axis=(1, 2, 3), keepdims=True)
    assert np.max(np.abs(cA - ref) / scale) < RTOL
    P.status()


def test_compress_non_uniform_rings():
    """Ring radii that are not equispaced (as from a Gauss-Jacobi rule) take the
    per-ring phase evaluation instead of the ring-to-ring rotation."""
    wl, A, B, U = setup(N=128, R=40, Q=256, N_B=2, N_A=3, T_side=3, H=12, seed=77)
    g = wl.grid
    rng = np.random.default_rng(3)
    k = np.sort(rng.uniform(1.0, g.K, size=g.R))
    w = rng.uniform(0.5, 2.0, size=g.R) * k
    At = torch.from_numpy(A).to(DEV)
    cA = P.compress(k, w, torch.from_numpy(U).to(DEV), At, deltas=wl.deltas).cpu().numpy()
    a_c = O.compress(O.translate(A.astype(np.complex128), k, wl.deltas), U, w)
    ref = pack_slots(a_c).reshape(3 * 9, 12, 128, 2)
    scale = np.max(np.abs(ref), axis=(1, 2, 3), keepdims=True)
    assert np.max(np.abs(cA - ref) / scale) < RTOL


@pytest.mark.parametrize("H", [32, 8])
def test_align_scores_tiny_workload(H):
    """64 images x 16 templates, 64x64 px, 32 rings, Q = 128, T = 1: full landscape."""
    wl, A, B, U = setup(N=64, R=32, Q=128, N_B=16, N_A=64, H=H, seed=0)
    cA, cB, T = _gpu(wl, A, B, U)
    X = P.align_scores(cA, 64, T, cB, 16, H, 128).cpu().numpy()
    Xr, _, _ = oracle_scores(wl, A, B, U)
    assert x_err(X, Xr) < RTOL
    assert frob_rel(X, Xr) < RTOL
    if H == 32:  # full rank also equals the uncompressed FB formula and the direct sum
        A_t = O.translate(A.astype(np.complex128), wl.grid.k, wl.deltas)
        Xd = O.scores_direct(A_t, B.astype(np.complex128), wl.grid.w).real
        assert x_err(X, Xd) < RTOL
    P.status()


def test_align_scores_with_translations_ragged():
    wl, A, B, U = setup(N=64, R=32, Q=256, N_B=5, N_A=3, T_side=3, H=12, seed=4)
    cA, cB, T = _gpu(wl, A, B, U)
    X = P.align_scores(cA, 3, T, cB, 5, 12, 256).cpu().numpy()
    Xr, _, _ = oracle_scores(wl, A, B, U)
    assert x_err(X, Xr) < RTOL


CASES = [
    # (Q, R, H, T_side, N_A, N_B)
    (128, 32, 8, 1, 64, 16),     # tiny workload, H = 8
    (128, 32, 32, 1, 64, 16),    # tiny workload, full rank
    (128, 32, 12, 1, 37, 23),    # ragged image groups and template batches
    (256, 64, 12, 3, 7, 13),     # throughput geometry, 9 translations, ragged
    (256, 64, 12, 3, 2, 1),      # single template
    (256, 64, 12, 3, 5, 4),      # one template batch, images spanning passes
    (256, 64, 8, 3, 11, 6),      # H = 8: nine passes per image group, two template batches
    (256, 64, 64, 2, 3, 5),      # H = 64 (widest register block), 4 translations
    (256, 40, 20, 1, 9, 11),     # H padded to 24
    (512, 48, 16, 2, 5, 4),      # Q = 512
    (512, 40, 12, 3, 9, 5),      # Q = 512, H = 12: two passes per image group, three template batches
    (512, 32, 7, 1, 13, 3),      # Q = 512, H padded to 8, ragged pass
    (512, 24, 16, 2, 3, 1300),   # Q = 512, 42.6 MB of templates: two template chunks across the grid
    (128, 24, 1, 1, 3, 3),       # H = 1
    (16, 6, 3, 1, 4, 3),         # Q = 16 (generic per-pair path)
    (1024, 20, 5, 1, 2, 3),      # Q = 1024 (generic per-pair path)
]


@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B", CASES)
def test_align_best_matches_oracle(Q, R, H, T_side, N_A, N_B):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=Q * 7 + H)
    cA, cB, T = _gpu(wl, A, B, U)
    Xr, _, _ = oracle_scores(wl, A, B, U)
    for pairwise in (False, True):
        best, arg, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=1.0, want_lse=True, pairwise=pairwise)
        check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)
        # without the log-sum-exp output
        b2, a2, _ = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=False, pairwise=pairwise)
        assert torch.equal(b2, best) and torch.equal(a2, arg)
    P.status()


@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B", [(256, 64, 12, 3, 7, 13), (256, 64, 16, 2, 5, 4),
                                                   (512, 48, 16, 2, 5, 4), (512, 40, 12, 3, 9, 5)])
def test_single_role_kernel_selection_matches_oracle(monkeypatch, Q, R, H, T_side, N_A, N_B):
    """RSVD_ALIGN_KERNEL=fused runs the single-role fused kernel where the
    warp-specialised one is the default (Q = 256, 512; H <= 16): same oracle
    bounds, and the same results as the default kernel up to rounding."""
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=Q * 5 + H)
    cA, cB, T = _gpu(wl, A, B, U)
    Xr, _, _ = oracle_scores(wl, A, B, U)
    ref = P.align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=1.0, want_lse=True)
    monkeypatch.setenv("RSVD_ALIGN_KERNEL", "fused")
    best, arg, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, inv_sigma2=1.0, want_lse=True)
    monkeypatch.delenv("RSVD_ALIGN_KERNEL")
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)
    scale = torch.clamp(ref[0].abs(), min=1e-30)
    assert float(((best - ref[0]).abs() / scale).max()) <= 2e-6
    P.status()


@pytest.mark.parametrize("inv_sigma2", [0.25, 4.0])
def test_lse_scale(inv_sigma2):
    wl, A, B, U = setup(N=128, R=64, Q=256, N_B=6, N_A=4, T_side=3, H=12, seed=9)
    cA, cB, T = _gpu(wl, A, B, U)
    Xr, _, _ = oracle_scores(wl, A, B, U)
    best, arg, lse = P.align_best(cA, 4, T, cB, 6, 12, 256, inv_sigma2=inv_sigma2, want_lse=True)
    check_best(Xr, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), inv_sigma2)


def test_noiseless_argmax_is_exact_and_recovers_truth():
    """Full rank on noiseless images made as T_{-delta_t0} R_{gamma_m0} B_j0: the
    GPU argmax equals the oracle's and the truth, and best = ||B_j0||^2."""
    from synthetic import make_workload, polar_norm2

    wl = make_workload(N=128, R=64, Q=256, N_B=6, N_A=10, snr=None, T_side=3, seed=11)
    A = wl.images.astype(np.complex64)
    B = wl.templates.astype(np.complex64)
    U, _ = O.principal_vectors(O.radial_kernel(B.astype(np.complex128), wl.grid.w), 64)
    cA, cB, T = _gpu(wl, A, B, U)
    Xr, _, _ = oracle_scores(wl, A, B, U)
    best, arg, _ = P.align_best(cA, 10, T, cB, 6, 64, 256)
    best, arg = best.cpu().numpy(), arg.cpu().numpy()
    mask = np.zeros((10, 6), dtype=bool)
    mask[np.arange(10), wl.truth_j] = True
    check_best(Xr, best, arg, exact_arg_mask=mask)
    for n in range(10):
        j = wl.truth_j[n]
        assert arg[n, j] == wl.truth_t[n] * 256 + wl.truth_m[n]
        nrm = polar_norm2(wl.grid, B[j].astype(np.complex128))
        assert abs(best[n, j] - nrm) < 1e-5 * nrm


@pytest.mark.parametrize("R,Q,N_B,H", [(32, 128, 16, 8), (64, 256, 200, 12), (128, 128, 40, 16), (7, 32, 5, 7)])
def test_build_radial_svd_matches_oracle(R, Q, N_B, H):
    from synthetic import make_workload

    wl = make_workload(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=1, snr=None, seed=R + N_B)
    B = wl.templates.astype(np.complex64)
    C = O.radial_kernel(B.astype(np.complex128), wl.grid.w)
    Ur, lam = O.principal_vectors(C, H)
    Ug, eg = P.build_radial_svd(wl.grid.w, torch.from_numpy(B).to(DEV), H)
    P.status()
    Ug, eg = Ug.cpu().numpy(), eg.cpu().numpy()
    assert np.max(np.abs(eg - lam)) <= 1e-10 * lam[0]
    # columns with a clear spectral gap agree including sign; the projector
    # onto the leading H vectors agrees when the H-th gap is clear
    ext = np.r_[np.inf, lam, -np.inf]
    gaps = np.minimum(ext[0:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
    for h in range(H):
        if gaps[h] > 1e-6 * lam[0]:
            assert np.max(np.abs(Ug[:, h] - Ur[:, h])) < 1e-6, h
    if H == R or lam[H - 1] - lam[H] > 1e-6 * lam[0]:
        assert np.max(np.abs(Ug @ Ug.T - Ur @ Ur.T)) < 1e-6
    assert np.allclose(Ug.T @ Ug, np.eye(H), atol=1e-10)


def test_throughput_workload_sampled_parity():
    """The 8192-image x 1024-template workload (128 px, 64 rings, Q = 256, 3x3
    translations, H = 12) on the GPU, in the launch configuration the
    benchmark times; 24 images x 16 templates of the output are checked
    against the oracle evaluated on exactly those objects."""
    from synthetic import CONFIGS, make_workload_torch

    cfg = CONFIGS["throughput"]
    grid, deltas, tmpl, imgs, truth = make_workload_torch(**cfg, seed=0, device=DEV)
    H = cfg["H"]
    U, eig = P.build_radial_svd(grid.w, tmpl, H)
    cA = P.compress(grid.k, grid.w, U, imgs, deltas=deltas)
    cB = P.compress(grid.k, grid.w, U, tmpl)
    T = deltas.shape[0]
    best, arg, lse = P.align_best(cA, cfg["N_A"], T, cB, cfg["N_B"], H, cfg["Q"], want_lse=True)
    P.status()
    rng = np.random.default_rng(1)
    ns = np.sort(rng.choice(cfg["N_A"], 24, replace=False))
    js = np.sort(rng.choice(cfg["N_B"], 16, replace=False))
    # include each sampled image's true template
    js = np.unique(np.concatenate([js, truth["j"][torch.from_numpy(ns).to(DEV)].cpu().numpy()]))
    A = imgs[torch.from_numpy(ns).to(DEV)].cpu().numpy().astype(np.complex128)
    B = tmpl[torch.from_numpy(js).to(DEV)].cpu().numpy().astype(np.complex128)
    Un = U.cpu().numpy()
    A_t = O.translate(A, grid.k, deltas)
    Xr = O.scores_compressed(O.compress(A_t, Un, grid.w), O.compress(B, Un, grid.w)).real
    b = best.cpu().numpy()[np.ix_(ns, js)]
    a = arg.cpu().numpy()[np.ix_(ns, js)]
    l_ = lse.cpu().numpy()[np.ix_(ns, js)]
    check_best(Xr, b, a, l_, 1.0)


def test_maximum_sizes_match_oracle():
    """The largest documented sizes together: R = 256 rings, H = 64 vectors,
    Q = 1024 angles, T = 64 translations (8 x 8 grid)."""
    R, Q, H = 256, 1024, 64
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=3, N_A=2, T_side=8, H=H, seed=31)
    cA, cB, T = _gpu(wl, A, B, U)
    assert T == 64
    best, arg, lse = P.align_best(cA, 2, T, cB, 3, H, Q, want_lse=True)
    P.status()
    X, _, _ = oracle_scores(wl, A, B, U)
    check_best(X, best.cpu().numpy(), arg.cpu().numpy(), lse.cpu().numpy(), 1.0)


@pytest.mark.gpu
def test_binding_rejects_short_buffers():
    """Operand and output buffers smaller than the call's sizes are refused by
    the binding (ValueError) before anything is launched."""
    N_A, T, N_B, H, Q = 3, 2, 4, 8, 128
    need_a = P.compressed_bytes(N_A, T, H, Q)
    cA = torch.zeros(need_a // 4 - 1, dtype=torch.float32, device=DEV)
    cB = torch.zeros(P.compressed_bytes(N_B, 1, H, Q) // 4, dtype=torch.float32, device=DEV)
    with pytest.raises(ValueError):
        P.align_best(cA, N_A, T, cB, N_B, H, Q)
    cA = torch.zeros(need_a // 4, dtype=torch.float32, device=DEV)
    with pytest.raises(ValueError):
        P.align_scores(cA, N_A, T, cB, N_B + 1, H, Q)
    best = torch.empty((N_A, N_B - 1), dtype=torch.float32, device=DEV)
    arg = torch.empty((N_A, N_B), dtype=torch.int32, device=DEV)
    with pytest.raises(ValueError):
        P.align_best(cA, N_A, T, cB, N_B, H, Q, out=(best, arg, None))
    with pytest.raises(ValueError):
        P.pack(cA, N_A, T + 1, H, Q, "bf16")
    P.status()
    b, a, _ = P.align_best(cA, N_A, T, cB, N_B, H, Q)  # the exact sizes pass
    P.status()
    assert b.shape == (N_A, N_B) and a.shape == (N_A, N_B)
