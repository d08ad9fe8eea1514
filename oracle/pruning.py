"""Felsenstein pruning in FP64 (oracle; test infrastructure only).

Follows the paper's statement of the problem: per-node partial likelihoods
computed in a post-order traversal (Sec. "Introduction": Felsenstein's
pruning algorithm), transition matrices P(t) from the rate matrix, cached
across patterns (Sec. "Discussion"), and the log-likelihood of the data at
the root. Readings where the paper is silent:

* partials are [category r, pattern p, state s] per node; a tip's partial is
  one-hot for a state code 0 <= c < S and all ones for any other code
  (ambiguous), the same in every category;
* P_r(t) = expm(rho_r * t * Q) -- computed with ``scipy.linalg.expm``, not
  the eigen formula the GPU path uses, so the two are independent;
* rescaling: at every internal node, each pattern's partial (all categories
  and states) is divided by 2^e where max = f * 2^e, f in [0.5, 1); the
  exponents are summed and added back as e * ln 2 at the root;
* the root distribution is the stationary pi; per-pattern likelihood is
  sum_r w_r sum_s pi_s p_root[r, p, s].
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

LN2 = float(np.log(2.0))


def transition_matrices(Q: np.ndarray, edge_len: np.ndarray, rates) -> np.ndarray:
    """P[v, r] = expm(rates[r] * edge_len[v] * Q) for every node v."""
    rates = np.asarray(rates, float)
    S = Q.shape[0]
    P = np.empty((len(edge_len), len(rates), S, S))
    for v, t in enumerate(edge_len):
        for r, rho in enumerate(rates):
            P[v, r] = expm(rho * t * Q)
    return P


def derivative_matrices(Q: np.ndarray, P: np.ndarray, rates) -> np.ndarray:
    """dP/dt for P = expm(rho t Q): rho * Q * P."""
    rates = np.asarray(rates, float)
    return np.einsum("r,ij,vrjk->vrik", rates, Q, P)


def tip_partials(states: np.ndarray, S: int) -> np.ndarray:
    """[n_tips, n_patterns, S] tip partials from int state codes."""
    states = np.asarray(states).astype(np.int64)
    out = np.zeros(states.shape + (S,))
    ok = (states >= 0) & (states < S)
    t_idx, p_idx = np.nonzero(ok)
    out[t_idx, p_idx, states[ok]] = 1.0
    out[~ok] = 1.0
    return out


def _rescale(x: np.ndarray):
    """Divide each pattern of x [R, P, S] by the power of two 2^e with
    max = f * 2^e, f in [0.5, 1). Returns (scaled, e)."""
    m = x.max(axis=(0, 2))
    _, e = np.frexp(m)
    e = np.where(m > 0, e, 0).astype(np.int64)
    return np.ldexp(x, -e[None, :, None]), e


def child_product(P_c: np.ndarray, p_c: np.ndarray) -> np.ndarray:
    """(P_c p_c)[r, p, i] = sum_j P_c[r, i, j] p_c[r, p, j]; a tip's p_c is
    [P, S] and is used in every category."""
    if p_c.ndim == 2:
        return np.einsum("rij,pj->rpi", P_c, p_c)
    return np.einsum("rij,rpj->rpi", P_c, p_c)


def post_order(children: np.ndarray, n_tips: int, P: np.ndarray,
               tips: np.ndarray, rescale: bool = True):
    """Post-order partials of every internal node.

    ``children[k]`` are the children of node n_tips + k, labelled so children
    come before parents; ``tips`` is [n_tips, P, S]. Returns (partials, exps)
    dicts keyed by node: partials [R, P, S] (rescaled if ``rescale``) and the
    per-pattern integer exponent removed at that node.
    """
    partials, exps = {}, {}

    def get(v):
        return tips[v] if v < n_tips else partials[v]

    for k, (a, b) in enumerate(np.asarray(children)):
        n = n_tips + k
        x = child_product(P[a], get(a)) * child_product(P[b], get(b))
        if rescale:
            x, e = _rescale(x)
        else:
            e = np.zeros(x.shape[1], dtype=np.int64)
        partials[n], exps[n] = x, e
    return partials, exps


def root_site_loglik(root_partial: np.ndarray, cum_exp: np.ndarray, pi,
                     cat_weights) -> np.ndarray:
    """l_p = log(sum_r w_r sum_s pi_s p_root[r, p, s]) + ln2 * E_p."""
    lik = np.einsum("r,s,rps->p", np.asarray(cat_weights, float),
                    np.asarray(pi, float), root_partial)
    with np.errstate(divide="ignore"):
        return np.log(lik) + LN2 * cum_exp


def loglik(tree, Q, pi, rates, cat_weights, pattern_weights, tip_states,
           rescale: bool = True, tip_partial_array=None):
    """(logL, site log-likelihoods) of ``tip_states`` [n_tips, P] on ``tree``
    (any object with n_tips, children and edge_len)."""
    S = Q.shape[0]
    P = transition_matrices(Q, tree.edge_len, rates)
    tips = tip_partial_array if tip_partial_array is not None else tip_partials(tip_states, S)
    partials, exps = post_order(tree.children, tree.n_tips, P, tips, rescale)
    root = 2 * tree.n_tips - 2
    cum = sum(exps.values())
    site = root_site_loglik(partials[root], cum, pi, cat_weights)
    return float(np.dot(pattern_weights, site)), site


def loglik_chunked(tree, Q, pi, rates, cat_weights, pattern_weights, tip_states,
                   chunk: int = 8192, patterns=None):
    """logL and site log-likelihoods over pattern chunks (patterns are
    conditionally independent given the tree, so chunks sum exactly). If
    ``patterns`` is given, only those pattern indices are evaluated."""
    S = Q.shape[0]
    P = transition_matrices(Q, tree.edge_len, rates)
    idx = np.arange(tip_states.shape[1]) if patterns is None else np.asarray(patterns)
    site = np.empty(len(idx))
    root = 2 * tree.n_tips - 2
    for lo in range(0, len(idx), chunk):
        sel = idx[lo:lo + chunk]
        tips = tip_partials(tip_states[:, sel], S)
        partials, exps = post_order(tree.children, tree.n_tips, P, tips, True)
        site[lo:lo + chunk] = root_site_loglik(partials[root], sum(exps.values()),
                                               pi, cat_weights)
    w = np.asarray(pattern_weights, float)[idx]
    return float(np.dot(w, site)), site
