"""Node-height ratio transform and its chain rule (oracle; test
infrastructure only).

Sec. "Algorithmic advances": node heights and branch-specific rates are
inferred together by a ratio transform of the node heights that keeps every
node older than its descendants. Readings: tips have fixed heights
(sampling times); each internal node v other than the root has an anchor
a_v, the largest tip height below it, and a ratio r_v in (0, 1) with
    h_v = a_v + r_v (h_parent(v) - a_v);
the root height is a free parameter; the branch above v has length
    t_v = rho_v (h_parent(v) - h_v)
in expected substitutions, rho_v its rate. The gradient with respect to
ratios, root height and rates follows from dlogL/dt by the chain rule,
written here directly from these definitions.
"""
from __future__ import annotations

import numpy as np


def parents(children, n_tips: int) -> np.ndarray:
    """parent[v] for every node (-1 at the root)."""
    children = np.asarray(children)
    par = -np.ones(2 * n_tips - 1, dtype=np.int64)
    for k, (a, b) in enumerate(children):
        par[a] = par[b] = n_tips + k
    return par


def anchors(children, n_tips: int, tip_height) -> np.ndarray:
    """a_v = the largest tip height in the subtree of v (tips: their own)."""
    a = np.empty(2 * n_tips - 1)
    a[:n_tips] = tip_height
    for k, (x, y) in enumerate(np.asarray(children)):
        a[n_tips + k] = max(a[x], a[y])
    return a


def heights(children, n_tips: int, tip_height, ratio, root_height) -> np.ndarray:
    """Node heights from tip heights, ratios (internal node n_tips + k ->
    ratio[k]; the root's entry unused) and the root height, root first."""
    par = parents(children, n_tips)
    anc = anchors(children, n_tips, tip_height)
    h = np.empty(2 * n_tips - 1)
    h[:n_tips] = tip_height
    root = 2 * n_tips - 2
    h[root] = root_height
    for v in range(root - 1, n_tips - 1, -1):      # parents before children
        h[v] = anc[v] + ratio[v - n_tips] * (h[par[v]] - anc[v])
    return h


def branch_lengths(children, n_tips: int, h, rate) -> np.ndarray:
    par = parents(children, n_tips)
    t = np.zeros(2 * n_tips - 1)
    for v in range(2 * n_tips - 2):
        t[v] = rate[v] * (h[par[v]] - h[v])
    return t


def ratio_gradient(children, n_tips: int, tip_height, ratio, root_height, rate, grad_len):
    """(dlogL/dratio [n_tips - 1] (root entry 0), dlogL/droot_height,
    dlogL/drate [2 n_tips - 1]) from dlogL/dt.

    dlogL/dh_v collects -rho_v g_v (the edge above v) and rho_c g_c for each
    child c; the total derivative G_v adds r_c G_c of every internal child
    (its height moves with h_v), children first; then dlogL/dr_v =
    (h_parent(v) - a_v) G_v, dlogL/drho_v = (h_parent(v) - h_v) g_v."""
    children = np.asarray(children)
    par = parents(children, n_tips)
    anc = anchors(children, n_tips, tip_height)
    h = heights(children, n_tips, tip_height, ratio, root_height)
    g = np.asarray(grad_len, float)
    root = 2 * n_tips - 2
    gh = np.zeros(2 * n_tips - 1)
    for v in range(n_tips, 2 * n_tips - 1):
        a, b = children[v - n_tips]
        gh[v] = rate[a] * g[a] + rate[b] * g[b] - (rate[v] * g[v] if v != root else 0.0)
    G = gh.copy()
    for v in range(n_tips, 2 * n_tips - 1):          # children before parents
        for c in children[v - n_tips]:
            if c >= n_tips:
                G[v] += ratio[c - n_tips] * G[c]
    gr = np.zeros(n_tips - 1)
    for v in range(n_tips, root):
        gr[v - n_tips] = (h[par[v]] - anc[v]) * G[v]
    grate = np.zeros(2 * n_tips - 1)
    for v in range(root):
        grate[v] = (h[par[v]] - h[v]) * g[v]
    return gr, G[root], grate
