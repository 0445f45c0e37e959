"""Host-input pipeline (rsvd_align_best_host): images and templates in host
memory, chunked copies overlapping compression and alignment. It runs the same
kernels as the device path, so results must match it exactly; the device path
itself is checked against the FP64 oracle in test_gpu_parity.py. One case is
also compared with the oracle directly."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.gpu_common import check_best, oracle_scores, setup  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"


def _device_path(wl, A, B, U, precision, want_lse):
    g = wl.grid
    T = wl.deltas.shape[0]
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(g.k, g.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas if T > 1 else None,
                    precision=precision)
    cB = P.compress(g.k, g.w, Ut, torch.from_numpy(B).to(DEV), precision=precision)
    H, Q = U.shape[1], g.Q
    best, arg, lse = P.align_best(cA, A.shape[0], T, cB, B.shape[0], H, Q, precision=precision, want_lse=want_lse)
    P.status()
    return best.cpu().numpy(), arg.cpu().numpy(), (lse.cpu().numpy() if want_lse else None)


@pytest.mark.parametrize("Q,R,H,T_side,N_A,N_B,chunk,precision,want_lse", [
    (256, 64, 12, 3, 37, 20, 16, "fp32", False),   # three chunks, ragged tail, T = 9
    (256, 64, 12, 3, 10, 7, 4, "fp32", True),      # with log-sum-exp
    (128, 32, 8, 1, 50, 16, 50, "fp32", False),    # one chunk
    (128, 32, 8, 1, 41, 9, 7, "bf16", False),      # tensor-core operands, six chunks
    (256, 64, 12, 3, 23, 6, 8, "fp16x3", True),    # row-scaled split: per-chunk compression, row factors
    (512, 48, 16, 2, 9, 5, 2, "fp32", False),      # Q = 512, T = 4
])
def test_host_pipeline_equals_device_path(Q, R, H, T_side, N_A, N_B, chunk, precision, want_lse):
    wl, A, B, U = setup(N=2 * R, R=R, Q=Q, N_B=N_B, N_A=N_A, T_side=T_side, H=H, seed=Q + N_A)
    g = wl.grid
    T = wl.deltas.shape[0]
    ref = _device_path(wl, A, B, U, precision, want_lse)
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    best, arg, lse = P.align_best_host(g.k, g.w, torch.from_numpy(U).to(DEV), Ah, Bh,
                                       deltas=wl.deltas if T > 1 else None, precision=precision,
                                       want_lse=want_lse, chunk=chunk)
    P.status()
    assert np.array_equal(best.numpy(), ref[0])
    assert np.array_equal(arg.numpy(), ref[1])
    if want_lse:
        assert np.array_equal(lse.numpy(), ref[2])


def test_host_pipeline_matches_oracle():
    wl, A, B, U = setup(N=128, R=64, Q=256, N_B=11, N_A=13, T_side=3, H=12, seed=5)
    g = wl.grid
    best, arg, _ = P.align_best_host(g.k, g.w, torch.from_numpy(U).to(DEV), torch.from_numpy(A).pin_memory(),
                                     torch.from_numpy(B).pin_memory(), deltas=wl.deltas, chunk=5)
    P.status()
    X, _, _ = oracle_scores(wl, A, B, U)
    check_best(X, best.numpy(), arg.numpy())


def test_host_pipeline_needs_two_streams():
    wl, A, B, U = setup(N=64, R=32, Q=128, N_B=2, N_A=3, T_side=1, H=4, seed=1)
    s = torch.cuda.current_stream()
    with pytest.raises(P.RSVDError):
        P.align_best_host(wl.grid.k, wl.grid.w, torch.from_numpy(U).to(DEV), torch.from_numpy(A),
                          torch.from_numpy(B), stream=s, copy_stream=s)
