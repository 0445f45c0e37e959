"""Multi-rank logic on CPU with the gloo backend (world size 2): image sharding,
row gathering, and the all-reduced template gradient of the log-sum-exp loss.
The per-rank compute is the FP64 oracle written as torch CPU ops (the CUDA
path needs a GPU); the sharding and collectives are the product's."""

import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2202_07235_gb300.parallel import shard


def test_shard_covers_every_item_once():
    for n in (0, 1, 7, 8192, 10001):
        for world in (1, 2, 3, 8):
            blocks = [shard(n, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == n
            for (a0, b0), (a1, b1) in zip(blocks, blocks[1:]):
                assert b0 == a1
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _torch_loss(images, templates, U, k, w, deltas, s):
    """L_n of the oracle's formulas in torch FP64 (differentiable)."""
    Q = images.shape[-1]
    psi = 2 * math.pi * torch.arange(Q, dtype=torch.float64) / Q
    k = torch.as_tensor(k)
    d = torch.as_tensor(deltas)
    ph = torch.exp(-1j * k[None, :, None] * (d[:, 0, None, None] * torch.cos(psi) + d[:, 1, None, None] * torch.sin(psi)))
    Wt = torch.as_tensor(U * np.sqrt(w)[:, None]).to(torch.complex128)
    a = torch.fft.fft(images[:, None] * ph[None], dim=-1) / Q
    b = torch.fft.fft(templates, dim=-1) / Q
    ac = torch.einsum("rh,ntrq->nthq", Wt, a)
    bc = torch.einsum("rh,jrq->jhq", Wt, b)
    X = torch.fft.fft(2 * math.pi * torch.einsum("nthq,jhq->ntjq", ac.conj(), bc), dim=-1).real
    return torch.logsumexp(X.reshape(X.shape[0], -1) * s, dim=1)


def _worker(rank, world, port, payload, out_q):
    import torch.distributed as dist

    from paper_2202_07235_gb300.parallel import distributed_lse_align, gather_rows

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, B, U, k, w, deltas, s = payload
        a0, a1 = shard(A.shape[0], rank, world)
        imgs = torch.tensor(A[a0:a1], requires_grad=True)
        tmpl = torch.tensor(B, requires_grad=True)
        L = distributed_lse_align(imgs, tmpl, lambda a, b: _torch_loss(a, b, U, k, w, deltas, s))
        L.sum().backward()
        L_all = gather_rows(L.detach(), A.shape[0])
        G_all = gather_rows(imgs.grad, A.shape[0])
        out_q.put((rank, L_all.numpy(), G_all.numpy(), tmpl.grad.numpy()))
    except Exception as e:  # report instead of leaving the parent waiting
        out_q.put((rank, repr(e), None, None))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.slow
def test_two_ranks_match_single_process_loss_and_gradients():
    import oracle as O
    from synthetic import make_workload

    wl = make_workload(N=32, R=12, Q=32, N_B=3, N_A=5, snr=0.1, T_side=3, seed=12)
    g = wl.grid
    U, _ = O.principal_vectors(O.radial_kernel(wl.templates, g.w), 6)
    s = 1.0
    loss, GA, GB = O.lse_loss_grad(wl.images, wl.templates, g.k, g.w, wl.deltas, U, s)
    payload = (wl.images, wl.templates, U, g.k, g.w, wl.deltas, s)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, payload, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    Ln = O.lse_loss(O.scores_compressed(O.compress(O.translate(wl.images, g.k, wl.deltas), U, g.w),
                                        O.compress(wl.templates, U, g.w)).real, s)[1]
    for rank, L_all, G_all, G_t in res:
        assert G_all is not None, L_all
        assert np.allclose(L_all, Ln, rtol=1e-12, atol=1e-12)
        assert np.allclose(G_all, GA, rtol=1e-10, atol=1e-12 * np.abs(GA).max())
        # the template gradient is the sum over both ranks' images
        assert np.allclose(G_t, GB, rtol=1e-10, atol=1e-12 * np.abs(GB).max())
