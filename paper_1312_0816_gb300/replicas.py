"""Data-parallel replicas: one process per GPU, each with its own copy of the
volume tables and its own share of the tracks.

The navigator step of Fig. 1 is evaluated per track, so the forward path
shards with no exchange at all: rank r handles its own baskets (shard() gives
a balanced contiguous split of a common basket; a generator seeded by rank
gives independent ones).  The one exchange is in the gradients: the geometry
gradients of the adjoint are sums over tracks, so a data-parallel backward adds
the per-rank sums.  They are a few doubles per daughter, so they are gathered
and added in rank order (allreduce_geometry), which keeps the result
bit-reproducible for a fixed number of ranks, unlike a ring sum.

Launch: `torchrun --nproc-per-node N` (RANK / LOCAL_RANK / WORLD_SIZE /
MASTER_ADDR / MASTER_PORT from the environment); backend "nccl" on GPUs,
"gloo" for CPU runs.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init(backend: str = "nccl", device=None) -> bool:
    """Joins the process group when more than one rank runs; returns whether
    it did."""
    import torch.distributed as tdist

    ws, _, _ = env()
    if ws <= 1 or tdist.is_initialized():
        return ws > 1
    if device is not None and backend == "nccl":
        tdist.init_process_group(backend, device_id=device)
    else:
        tdist.init_process_group(backend)
    return True


def active() -> bool:
    import torch.distributed as tdist

    return tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1


def shard(n_total: int, world: int, rank: int):
    """(offset, count) of rank's contiguous share of n_total tracks; the first
    n_total % world ranks take one more."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(n_total, world)
    count = q + (1 if rank < r else 0)
    offset = rank * q + min(rank, r)
    return offset, count


def barrier():
    import torch.distributed as tdist

    if active():
        tdist.barrier()


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value over the ranks (a timing: the slowest rank's)."""
    import torch
    import torch.distributed as tdist

    if not active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device="cpu") -> float:
    import torch
    import torch.distributed as tdist

    if not active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.SUM)
    return float(t.item())


def allreduce_geometry(*grads):
    """Adds each geometry-gradient tensor over the ranks, in place, in rank
    order: every rank gathers all ranks' copies and sums them 0, 1, ..., so
    all ranks hold the same bits and a rerun reproduces them."""
    import torch
    import torch.distributed as tdist

    if not active():
        return grads
    ws = tdist.get_world_size()
    for g in grads:
        if g is None:
            continue
        flat = g.contiguous().reshape(-1)
        parts = [torch.empty_like(flat) for _ in range(ws)]
        tdist.all_gather(parts, flat)
        acc = parts[0].clone()
        for r in range(1, ws):
            acc += parts[r]
        g.copy_(acc.reshape(g.shape))
    return grads
