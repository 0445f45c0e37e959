"""The allocation-free build entry point (for callers that cannot allocate
device scratch: plugins handed raw pointers, services with a fixed device
footprint) against the workspace entry point, through the C ABI.

Kept in a file that pytest collects last, so a run stopped at the first
failure has already run every other test."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_2202_07235_gb300 as P  # noqa: E402
from synthetic import make_workload  # noqa: E402


def _compare(Ua, ea, Ub, eb):
    """Same tolerance as the oracle parity of the build: eigenvalues to 1e-10 of the
    largest, columns with a clear spectral gap to 1e-6."""
    Ua, ea, Ub, eb = (x.cpu().numpy() for x in (Ua, ea, Ub, eb))
    assert np.max(np.abs(ea - eb)) <= 1e-10 * eb[0]
    H = Ua.shape[1]
    ext = np.r_[np.inf, eb, -np.inf]
    gaps = np.minimum(ext[0:H] - ext[1:H + 1], ext[1:H + 1] - ext[2:H + 2])
    for h in range(H):
        if gaps[h] > 1e-6 * eb[0]:
            assert np.max(np.abs(Ua[:, h] - Ub[:, h])) < 1e-6, h


def test_noalloc_build_matches_workspace_build_on_two_calls_in_a_row():
    cases = [dict(N=256, R=128, Q=128, N_B=40, H=16, seed=3), dict(N=128, R=64, Q=256, N_B=200, H=12, seed=5)]
    for c in cases:  # two calls in a row on the shared scratch, different sizes
        wl = make_workload(N=c["N"], R=c["R"], Q=c["Q"], N_B=c["N_B"], N_A=1, snr=None, seed=c["seed"])
        B = torch.from_numpy(wl.templates.astype(np.complex64)).to("cuda:0")
        U_ref, e_ref = P.build_radial_svd(wl.grid.w, B, c["H"])
        U_na, e_na = P.build_radial_svd_noalloc(wl.grid.w, B, c["H"])
        P.status()
        _compare(U_na, e_na, U_ref, e_ref)
        # and directly against the FP64 oracle on the same (complex64) templates
        C = O.radial_kernel(wl.templates.astype(np.complex64).astype(np.complex128), wl.grid.w)
        U_o, e_o = O.principal_vectors(C, c["H"])
        _compare(U_na, e_na, torch.from_numpy(U_o), torch.from_numpy(e_o))


def test_noalloc_build_largest_grid_fits_exactly():
    """R = 181 is the largest grid whose four R x R FP64 matrices fit the 1 MiB
    scratch (4 x 262,144 bytes, one template slice)."""
    wl = make_workload(N=362, R=181, Q=16, N_B=3, N_A=1, snr=None, seed=2)
    B = torch.from_numpy(wl.templates.astype(np.complex64)).to("cuda:0")
    U_na, e_na = P.build_radial_svd_noalloc(wl.grid.w, B, 4)
    P.status()
    U_ref, e_ref = P.build_radial_svd(wl.grid.w, B, 4)
    _compare(U_na, e_na, U_ref, e_ref)
    C = O.radial_kernel(wl.templates.astype(np.complex64).astype(np.complex128), wl.grid.w)
    U_o, e_o = O.principal_vectors(C, 4)
    _compare(U_na, e_na, torch.from_numpy(U_o), torch.from_numpy(e_o))


@pytest.mark.parametrize("R", [182, 192])
def test_noalloc_build_rejects_grids_beyond_its_scratch(R):
    from paper_2202_07235_gb300._native import RSVDError

    wl = make_workload(N=2 * R, R=R, Q=32, N_B=2, N_A=1, snr=None, seed=1)
    B = torch.from_numpy(wl.templates.astype(np.complex64)).to("cuda:0")
    with pytest.raises(RSVDError) as e:
        P.build_radial_svd_noalloc(wl.grid.w, B, 4)
    assert e.value.code == -2
