"""Failure detection without a GPU fault: a device-side wait that can never
complete gives up after its clock budget, records RSVD_ETIMEOUT in the status
word, and the context stays usable for the next call."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests.gpu_common import check_best, oracle_scores, setup  # noqa: E402

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2202_07235_gb300 as P  # noqa: E402

DEV = "cuda:0"
RSVD_ETIMEOUT = -5


def test_bounded_wait_gives_up_and_reports_timeout():
    P.status()  # nothing pending
    assert P.selftest_wait_timeout(1 << 21) == RSVD_ETIMEOUT  # about a millisecond of waiting
    P.status()  # read and cleared: the next check is clean
    # the context is still usable: a small alignment matches the oracle
    wl, A, B, U = setup(N=64, R=32, Q=128, N_B=3, N_A=4, T_side=1, H=8, seed=5)
    Ut = torch.from_numpy(U).to(DEV)
    cA = P.compress(wl.grid.k, wl.grid.w, Ut, torch.from_numpy(A).to(DEV), deltas=wl.deltas)
    cB = P.compress(wl.grid.k, wl.grid.w, Ut, torch.from_numpy(B).to(DEV))
    best, arg, _ = P.align_best(cA, 4, 1, cB, 3, 8, 128)
    P.status()
    X, _, _ = oracle_scores(wl, A, B, U)
    check_best(X, best.cpu().numpy(), arg.cpu().numpy())


def test_timeouts_are_reported_once_per_failure():
    for _ in range(3):
        assert P.selftest_wait_timeout(1 << 16) == RSVD_ETIMEOUT
    assert int(P.lib().rsvd_status(torch.cuda.current_stream().cuda_stream)) == 0
