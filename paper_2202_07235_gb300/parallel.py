"""Multi-GPU use: one process per GPU, images sharded, templates replicated.

Scoring is independent per (image, template) pair, so the forward pass needs
no collective: each rank compresses and aligns its own contiguous block of
images against all templates (weak scaling). The exchange steps are:

* the template gradient of the log-sum-exp loss, a sum over all images, is
  all-reduced (sum) across ranks after each rank's rsvd_lse_backward;
* the per-image normalisers L_n stay on the rank that owns the image.

torch.distributed (NCCL on GPUs, gloo on CPU) carries the collectives; no
arithmetic of the method happens here.
"""

from __future__ import annotations

import torch


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous balanced block [start, stop) of n items owned by `rank`."""
    if world <= 0 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    stop = start + base + (1 if rank < extra else 0)
    return start, stop


def allreduce_sum_(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over ranks (no-op when torch.distributed is not initialised)."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def gather_rows(t: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """Concatenate per-rank row blocks (in rank order, as produced by `shard`)."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return t
    world = dist.get_world_size(group)
    blocks = [shard(n_total, r, world) for r in range(world)]
    width = max(b - a for a, b in blocks)  # collectives need equal sizes: pad, then trim
    padded = torch.zeros((width,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    padded[: t.shape[0]] = t
    parts = [torch.empty_like(padded) for _ in blocks]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, blocks)], dim=0)


class DistributedLSEAlign(torch.autograd.Function):
    """Log-sum-exp alignment loss over images sharded across ranks: forward is
    the local LSEAlign on this rank's images; backward all-reduces the template
    gradient (images' gradients stay local). `local_fn(images, templates)`
    computes the local per-image loss with autograd (e.g. api.lse_align bound to
    U, k, w, deltas, sigma)."""

    @staticmethod
    def forward(ctx, images, templates, local_fn, group):
        with torch.enable_grad():
            a = images.detach().requires_grad_(True)
            b = templates.detach().requires_grad_(True)
            L = local_fn(a, b)
        ctx.save_for_backward(a, b, L)
        ctx.group = group
        return L.detach()

    @staticmethod
    def backward(ctx, gL):
        a, b, L = ctx.saved_tensors
        ga, gb = torch.autograd.grad(L, (a, b), gL)
        allreduce_sum_(gb, ctx.group)
        return ga, gb, None, None


def distributed_lse_align(images, templates, local_fn, group=None):
    return DistributedLSEAlign.apply(images, templates, local_fn, group)
