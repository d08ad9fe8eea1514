"""Likelihood by its definition (oracle; test infrastructure only).

L_p = sum_r w_r sum over every assignment x of states to the internal nodes
of pi[x_root] * prod over edges (v above w) P_r(t_w)[x_v, x_w], with a tip's
state summed against its tip partial. Exponential in the number of internal
nodes: for trees of at most 6 taxa (4 states) or 3 taxa (61 states).
"""
from __future__ import annotations

import itertools

import numpy as np


def site_likelihood(children, n_tips, P, pi, cat_weights, tips):
    """Per-pattern likelihood [P] by enumerating internal states.

    ``P[v, r]`` is the matrix on the edge above v; ``tips`` [n_tips, P, S]."""
    children = np.asarray(children)
    n_int = n_tips - 1
    S = P.shape[-1]
    R = P.shape[1]
    pi = np.asarray(pi, float)
    cw = np.asarray(cat_weights, float)
    # tip factor: for tip c under internal state x of its parent,
    # T_c[r, p, x] = sum_s P_c[r, x, s] tips[c, p, s]
    tipf = {c: np.einsum("rxs,ps->rpx", P[c], tips[c]) for c in range(n_tips)}
    n_pat = tips.shape[1]
    total = np.zeros((R, n_pat))
    root = 2 * n_tips - 2
    for x in itertools.product(range(S), repeat=n_int):
        state = {n_tips + k: x[k] for k in range(n_int)}
        term = np.full((R, n_pat), pi[state[root]])
        for k, (a, b) in enumerate(children):
            n = n_tips + k
            for c in (a, b):
                if c < n_tips:
                    term = term * tipf[c][:, :, state[n]]
                else:
                    term = term * P[c][:, state[n], state[c]][:, None]
        total += term
    return np.einsum("r,rp->p", cw, total)
