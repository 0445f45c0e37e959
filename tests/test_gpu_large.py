"""The large workload (65,536 images of 256 px x 4,096 templates, 128 rings,
Q = 512, 5 x 5 translations, H = 16) at full size, in the launch configuration
the benchmark times: sampled outputs checked against the FP64 oracle evaluated
on exactly those objects. Its log-sum-exp gradient is checked at the same
geometry with fewer objects."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from tests.gpu_common import check_best, pack_slots  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402
from synthetic import CONFIGS, make_workload_torch  # noqa: E402

DEV = "cuda:0"


def test_large_workload_sampled_parity():
    cfg = CONFIGS["large"]
    N_A, N_B, Q, H = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["H"]
    grid, deltas, tmpl, imgs, truth = make_workload_torch(**cfg, seed=0, device=DEV)
    T = deltas.shape[0]
    rng = np.random.default_rng(2)
    ns = np.sort(rng.choice(N_A, 8, replace=False))
    js = np.sort(rng.choice(N_B, 16, replace=False))
    idx = torch.from_numpy(ns).to(DEV)
    js = np.unique(np.concatenate([js, truth["j"][idx].cpu().numpy()]))
    A = imgs[idx].cpu().numpy().astype(np.complex128)
    B = tmpl[torch.from_numpy(js).to(DEV)].cpu().numpy().astype(np.complex128)
    U, _ = P.build_radial_svd(grid.w, tmpl, H)
    cA = P.compress(grid.k, grid.w, U, imgs, deltas=deltas)
    del imgs
    torch.cuda.empty_cache()
    cB = P.compress(grid.k, grid.w, U, tmpl)
    best, arg, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=True)
    P.status()
    Un = U.cpu().numpy()
    Xr = O.scores_compressed(O.compress(O.translate(A, grid.k, deltas), Un, grid.w), O.compress(B, Un, grid.w)).real
    sel = np.ix_(ns, js)
    check_best(Xr, best.cpu().numpy()[sel], arg.cpu().numpy()[sel], lse.cpu().numpy()[sel], 1.0)


def test_large_geometry_gradient():
    cfg = {**CONFIGS["large"], "N_A": 40, "N_B": 96}
    N_A, N_B, Q, H = cfg["N_A"], cfg["N_B"], cfg["Q"], cfg["H"]
    grid, deltas, tmpl, imgs, _ = make_workload_torch(**cfg, seed=5, device=DEV)
    T = deltas.shape[0]
    U, _ = P.build_radial_svd(grid.w, tmpl, H)
    cA = P.compress(grid.k, grid.w, U, imgs, deltas=deltas)
    cB = P.compress(grid.k, grid.w, U, tmpl)
    _, _, lse = P.align_best(cA, N_A, T, cB, N_B, H, Q, want_lse=True)
    L = P.lse_rows(lse)
    gA, gB = P.lse_backward(cA, N_A, T, cB, N_B, H, Q, 1.0, L, torch.ones(N_A, dtype=torch.float32, device=DEV))
    P.status()
    ns = np.array([0, 17, 39])
    idx = torch.from_numpy(ns).to(DEV)
    Un = U.cpu().numpy()
    a_c = O.compress(O.translate(imgs[idx].cpu().numpy().astype(np.complex128), grid.k, deltas), Un, grid.w)
    b_c = O.compress(tmpl.cpu().numpy().astype(np.complex128), Un, grid.w)
    _, Ln, G_ac, _ = O.lse_grad_compressed(a_c, b_c, 1.0)
    assert np.max(np.abs(L[idx].cpu().numpy() - Ln)) < 1e-5 * np.max(np.abs(Ln))
    got = gA.view(N_A, T, H, Q // 2, 2)[idx].cpu().numpy()
    ref = pack_slots(G_ac)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < 5e-5
