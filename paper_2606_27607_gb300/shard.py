"""Pattern-block sharding across processes (one instance per GPU).

Patterns are conditionally independent given the tree, so an alignment
splits into blocks evaluated by separate instances with no exchange during a
traversal (Sec. "Benchmarks on NVIDIA and AMD GPUs": one instance per GPU over
conditionally independent blocks). The only combination step is a sum of the
per-block log-likelihoods and gradients.
"""
from __future__ import annotations

import numpy as np


def pattern_blocks(n_patterns: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [lo, hi) blocks whose sizes differ by at most one."""
    if world < 1:
        raise ValueError("world >= 1")
    base, extra = divmod(n_patterns, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def allreduce_sum(values: np.ndarray, group=None) -> np.ndarray:
    """Sum a float64 vector over the ranks of ``group`` (torch.distributed)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()
