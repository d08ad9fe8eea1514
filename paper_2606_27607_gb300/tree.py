"""Operation lists for a rooted binary tree (index bookkeeping only).

A tree is given as ``children`` ([N-1, 2] array: children of internal node
N+k, children before parents) and ``n_tips``; node v's buffer index is v and
the matrix slot of the edge above v is v (P) or n_nodes + v (dP/dt). The
pre-order partial of internal node v lives in buffer ``pre_base + v``.
"""
from __future__ import annotations

import numpy as np

from ._lib import ADJ_OP_DTYPE, EDGE_DTYPE, EIG_OP_DTYPE, OP_DTYPE, PRE_OP_DTYPE


def n_nodes(n_tips: int) -> int:
    return 2 * n_tips - 1


def post_ops(children, n_tips: int) -> np.ndarray:
    """Post-order partials updates, one per internal node (children first)."""
    children = np.asarray(children)
    ops = np.zeros(len(children), dtype=OP_DTYPE)
    for k, (a, b) in enumerate(children):
        ops[k] = (n_tips + k, a, a, b, b)
    return ops


def pre_ops(children, n_tips: int, pre_base: int, with_edges: bool = True,
            tip_pre: bool = False) -> np.ndarray:
    """Pre-order ops, one per internal node, root first. ``edge`` slots are
    node indices; q of internal node v goes to buffer pre_base + v (tips too
    when ``tip_pre``)."""
    children = np.asarray(children)
    N = n_tips
    root = 2 * N - 2
    nn = n_nodes(N)
    ops = np.zeros(N - 1, dtype=PRE_OP_DTYPE)
    for i, v in enumerate(range(root, N - 1, -1)):
        a, b = children[v - N]
        parent_pre = -1 if v == root else pre_base + v
        pre = [pre_base + c if (c >= N or tip_pre) else -1 for c in (a, b)]
        edge = [a, b] if with_edges else [-1, -1]
        ops[i] = (parent_pre, (a, b), (a, b), (nn + a, nn + b), pre, edge)
    return ops


def eig_ops(children, n_tips: int, edge_len) -> np.ndarray:
    """Post-order ops carrying their children's edge lengths (matrices formed
    on the fly)."""
    children = np.asarray(children)
    ops = np.zeros(len(children), dtype=EIG_OP_DTYPE)
    for k, (a, b) in enumerate(children):
        ops[k] = (n_tips + k, a, b, 0, edge_len[a], edge_len[b])
    return ops


def q_ops(children, n_tips: int, pre_base: int) -> np.ndarray:
    """Pre-order ops that only store q of every internal node (no edges, no
    derivative matrices): the input of the adjoint."""
    ops = pre_ops(children, n_tips, pre_base, with_edges=False)
    ops["dmat"] = -1
    return ops


def adj_ops(children, n_tips: int, pre_base: int) -> np.ndarray:
    """Adjoint ops, one per internal node: its post-order buffer, its q
    buffer (-1 at the root), both children, their edges' matrix slots and
    output slots (node indices)."""
    children = np.asarray(children)
    N = n_tips
    root = 2 * N - 2
    ops = np.zeros(N - 1, dtype=ADJ_OP_DTYPE)
    for k, (a, b) in enumerate(children):
        v = N + k
        ops[k] = (v, -1 if v == root else pre_base + v, (a, b), (a, b), (a, b))
    return ops


def edges(n_tips: int, pre_base: int) -> np.ndarray:
    """Every non-root edge for tl_edge_derivatives (pre buffers for all nodes)."""
    nn = n_nodes(n_tips)
    e = np.zeros(nn - 1, dtype=EDGE_DTYPE)
    for v in range(nn - 1):
        e[v] = (v, pre_base + v, v)
    return e
