"""Replica runs on several GPUs of one node.

The solve and the force do not shard (one lattice per GPU), so N GPUs run N
independent replicas: one process per GPU (launched by torchrun, which sets
RANK / LOCAL_RANK / WORLD_SIZE / MASTER_ADDR / MASTER_PORT), a barrier around
the timed region and the maximum of the ranks' times.  No data-path
collective exists."""
from __future__ import annotations

import os

import torch


def env():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl"):
    """Join the process group when more than one rank runs."""
    _, world, _ = env()
    if world > 1 and not torch.distributed.is_initialized():
        torch.distributed.init_process_group(backend)


def active() -> bool:
    return torch.distributed.is_available() and torch.distributed.is_initialized()


def barrier():
    if active():
        torch.distributed.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over all ranks (x itself on a single rank)."""
    if not active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def finalize():
    if active():
        torch.distributed.destroy_process_group()
