"""Subtree checkpointing: logL and its branch-length gradient with post-order
partials kept only at checkpoint depths, the rest recomputed during the
pre-order pass (for trees whose partials exceed device memory).

The tree is cut into bands of ``band`` consecutive depths below the root.
Post-order partials of the nodes at the top depth of every band (the
checkpoints) are kept; the other internal nodes of a band live in buffers
that are reused from band to band. Forward: bands bottom-up, one post-order
call each (a band's children are its own nodes, the checkpoints of the band
below, or tips). Backward: bands top-down; each band's non-checkpoint
partials are recomputed from the checkpoints below it, then one fused
pre-order + gradient call runs the band's parents, reading the q of the
band's top depth written by the band above and writing the q of the next
band's top depth. Every edge's derivative comes from its parent's op, so the
gradient is the same arithmetic as one whole-tree pass (the tests require
bit-identical results). Cost: one extra post-order pass. Memory: checkpoint
buffers plus two bands of reusable buffers instead of 2(N - 1).

All device work runs in the library; this module assigns buffers and builds
op lists (Sec. "Algorithmic advances": the pre-order traversal reads every
node's post-order partial once).
"""
from __future__ import annotations

import numpy as np

from ._lib import OP_DTYPE, PRE_OP_DTYPE, Instance


def depths(children, n_tips: int) -> np.ndarray:
    """Depth below the root of every node (root 0); internal nodes are
    numbered after their children, so a decreasing sweep sees parents
    first."""
    children = np.asarray(children)
    nn = 2 * n_tips - 1
    d = np.zeros(nn, dtype=np.int64)
    for v in range(nn - 1, n_tips - 1, -1):
        for c in children[v - n_tips]:
            d[c] = d[v] + 1
    return d


def layout(children, n_tips: int, band: int) -> dict:
    """Checkpoint set, bands and buffer counts for a band length (no device
    work): ``n_buffers`` internal buffers replace the 2 (N - 1) of the
    whole-tree layout."""
    children = np.asarray(children)
    band = max(1, int(band))
    d = depths(children, n_tips)
    internal = np.arange(n_tips, 2 * n_tips - 1)
    bandof = d // band
    ckpt = {int(v) for v in internal if d[v] % band == 0}
    n_bands = int(bandof[internal].max()) + 1
    bands = [[int(v) for v in internal if bandof[v] == b] for b in range(n_bands)]
    tr_size = max(sum(1 for v in b if v not in ckpt) for b in bands)
    q_size = max(len(b) + sum(1 for v in internal if bandof[v] == k + 1 and int(v) in ckpt)
                 for k, b in enumerate(bands))
    return dict(band=band, depth=d, bandof=bandof, ckpt=ckpt, bands=bands, tr_size=tr_size,
                q_size=q_size, n_buffers=len(ckpt) + tr_size + q_size)


def best_band(children, n_tips: int, candidates=(2, 3, 4, 6, 8)) -> tuple[int, int]:
    """(band, internal buffers) of the candidate band length needing the
    fewest buffers."""
    return min(((b, layout(children, n_tips, b)["n_buffers"]) for b in candidates),
               key=lambda x: (x[1], x[0]))


class CheckpointedLikelihood:
    """One tree on one instance, post-order partials kept at checkpoint
    depths 0, band, 2 band, ... (internal nodes only)."""

    def __init__(self, n_tips: int, n_patterns: int, children, n_states: int = 4,
                 n_categories: int = 4, precision: str = "f32", band: int = 4,
                 stream: int | None = None, create: bool = True):
        self.N, self.nn = n_tips, 2 * n_tips - 1
        self.children = np.asarray(children)
        lay = layout(self.children, n_tips, band)
        self.band, self.depth, self.bandof = lay["band"], lay["depth"], lay["bandof"]
        self.ckpt, self.bands = lay["ckpt"], lay["bands"]
        # buffers: one per checkpoint, a reusable pool for a band's other
        # nodes, and q buffers for a band's internal nodes plus the next
        # band's top depth
        self.ck_buf = {}
        nxt = n_tips
        for v in sorted(self.ckpt):
            self.ck_buf[v] = nxt
            nxt += 1
        self.tr_base, self.tr_size = nxt, lay["tr_size"]
        nxt += self.tr_size
        self.q_base, self.q_size = nxt, lay["q_size"]
        nxt += self.q_size
        self.n_buffers = nxt - n_tips
        self.inst = None
        if create:   # create=False: the op lists only (no device)
            self.inst = Instance(n_tips, n_patterns, n_states, n_categories, self.n_buffers,
                                 2 * self.nn, 1, precision, True, stream)
        self._plan()

    def close(self):
        if self.inst is not None:
            self.inst.close()

    # ---- buffer plan ------------------------------------------------------
    def _plan(self):
        N = self.N
        self.post_ops, self.re_ops, self.pre_ops = [], [], []
        q_of_top = {}      # q buffer of each checkpoint node (written by the band above)
        for b, nodes in enumerate(self.bands):
            tr = {v: self.tr_base + i for i, v in enumerate(x for x in nodes if x not in self.ckpt)}

            def post_buf(v):
                if v < N:
                    return v
                return self.ck_buf[v] if v in self.ckpt else tr[v]

            ops = np.zeros(len(nodes), dtype=OP_DTYPE)
            for i, v in enumerate(sorted(nodes)):          # children first
                a, c = self.children[v - N]
                ops[i] = (post_buf(v), post_buf(a), a, post_buf(c), c)
            self.post_ops.append(ops)
            self.re_ops.append(ops[[post_buf(v) >= self.tr_base for v in sorted(nodes)]])
            # pre-order: parents of this band, root first (decreasing labels)
            qb = {}
            for v in nodes:
                if v in q_of_top:
                    qb[v] = q_of_top[v]
            q_of_top_next = {}
            pre = np.zeros(len(nodes), dtype=PRE_OP_DTYPE)
            used = set(qb.values())
            free = [x for x in range(self.q_base, self.q_base + self.q_size) if x not in used]
            for i, v in enumerate(sorted(nodes, reverse=True)):
                a, c = self.children[v - N]
                parent_pre = -1 if v == self.nn - 1 else qb[v]
                outs = []
                for ch in (a, c):
                    if ch < N:
                        outs.append(-1)
                        continue
                    buf = free.pop(0)
                    if self.bandof[ch] == b:
                        qb[ch] = buf
                    else:
                        q_of_top_next[ch] = buf
                    outs.append(buf)
                pre[i] = (parent_pre, (post_buf(a), post_buf(c)), (a, c),
                          (self.nn + a, self.nn + c), outs, (a, c))
            self.pre_ops.append(pre)
            q_of_top = q_of_top_next

    # ---- evaluation -------------------------------------------------------
    def set_data(self, tips, model: str, params, freqs, rates, weights=None,
                 pattern_weights=None):
        for t in range(self.N):
            self.inst.set_tip_states(t, tips[t])
        self.inst.set_model(0, model, params, freqs)
        self.inst.set_category_rates(rates)
        if weights is not None:
            self.inst.set_category_weights(weights)
        if pattern_weights is not None:
            self.inst.set_pattern_weights(pattern_weights)

    def loglik(self, edge_len) -> float:
        """logL: the banded post-order pass (no derivative matrices)."""
        v = np.arange(self.nn - 1, dtype=np.int32)
        self.inst.update_matrices(0, v, np.asarray(edge_len, float)[: self.nn - 1], None)
        for b in range(len(self.bands) - 1, -1, -1):
            self.inst.update_partials(self.post_ops[b])
        return self.inst.root_loglik(self.ck_buf[self.nn - 1], 0)

    def n_bands(self) -> int:
        return len(self.bands)

    def launch(self, edge_len, gradient: bool, out_ptr: int) -> None:
        """Queue one evaluation on the instance's stream without waiting:
        logL to the device double at out_ptr and, with ``gradient``, band b's
        share of dlogL/dt (2N - 1 doubles, zeros outside the band) at
        out_ptr + 8 (1 + b (2N - 1)); the gradient is the sum of the band
        vectors (every edge appears in exactly one)."""
        v = np.arange(self.nn - 1, dtype=np.int32)
        el = np.asarray(edge_len, float)[: self.nn - 1]
        self.inst.update_matrices(0, v, el, (self.nn + v).astype(np.int32) if gradient else None)
        for b in range(len(self.bands) - 1, -1, -1):
            self.inst.update_partials(self.post_ops[b])
        self.inst.root_loglik_dev(self.ck_buf[self.nn - 1], 0, out_ptr)
        if not gradient:
            return
        for b in range(len(self.bands)):
            if b > 0 and len(self.re_ops[b]):
                self.inst.update_partials(self.re_ops[b])
            self.inst.pre_order_gradient_dev(self.pre_ops[b], self.nn, 0,
                                             out_ptr + 8 * (1 + b * self.nn))

    def gradient(self, edge_len):
        """(logL, dlogL/dt for every node (root 0)) with checkpointing."""
        v = np.arange(self.nn - 1, dtype=np.int32)
        self.inst.update_matrices(0, v, np.asarray(edge_len, float)[: self.nn - 1],
                                  (self.nn + v).astype(np.int32))
        for b in range(len(self.bands) - 1, -1, -1):     # forward, bottom-up
            self.inst.update_partials(self.post_ops[b])
        logl = self.inst.root_loglik(self.ck_buf[self.nn - 1], 0)
        g = np.zeros(self.nn)
        for b in range(len(self.bands)):                 # backward, top-down
            if b > 0 and len(self.re_ops[b]):
                self.inst.update_partials(self.re_ops[b])
            g += self.inst.pre_order_gradient(self.pre_ops[b], self.nn, 0)
        return logl, g
