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


class ChunkedLikelihood:
    """One tree whose patterns are evaluated in consecutive blocks on one
    instance sized for the largest block (the partials of all patterns need
    not fit at once). Each evaluation uploads every block's tip states and
    pattern weights before its passes; logL and the gradient are the sums
    over blocks (patterns are conditionally independent given the tree)."""

    def __init__(self, n_tips: int, n_patterns: int, n_blocks: int, n_states: int = 4,
                 n_categories: int = 4, precision: str = "f32", stream: int | None = None):
        from . import TreeLikelihood
        self.blocks = pattern_blocks(n_patterns, n_blocks)
        self.width = max(hi - lo for lo, hi in self.blocks)
        self.tl = TreeLikelihood(n_tips, self.width, n_states, n_categories, precision, stream)

    def close(self):
        self.tl.close()

    def set_data(self, tips, model: str, params, freqs, rates, weights=None,
                 pattern_weights=None):
        self.tips = np.asarray(tips)
        self.pw = (np.ones(self.tips.shape[1]) if pattern_weights is None
                   else np.asarray(pattern_weights, float))
        self.tl.set_model(model, params, freqs)
        self.tl.set_rates(rates, weights)

    def _block(self, lo: int, hi: int) -> None:
        n = hi - lo
        tips = np.full((self.tips.shape[0], self.width), -1, dtype=np.int8)
        tips[:, :n] = self.tips[:, lo:hi]
        w = np.zeros(self.width)
        w[:n] = self.pw[lo:hi]          # the unused tail of the last block weighs 0
        self.tl.inst.set_tip_states_all(tips)
        self.tl.set_pattern_weights(w)

    def gradient(self, children, edge_len):
        """(logL, dlogL/dt per node) summed over the blocks."""
        self.tl.set_tree(children, edge_len)
        logl, g = 0.0, None
        for lo, hi in self.blocks:
            self._block(lo, hi)
            lb, gb = self.tl.gradient()
            logl += lb
            g = gb if g is None else g + gb
        return logl, g
