"""Pre-order partials and log-likelihood gradients in FP64 (oracle; test
infrastructure only).

The paper's linear-time gradient (Sec. "Algorithmic advances") complements
the post-order traversal with a pre-order traversal; the likelihood is the
inner product of post- and pre-order partials at any node, and the gradient
w.r.t. every branch-length parameter follows in one pre-order pass through
the sandwich of a pre-order partial, the rate matrix and a post-order
partial (Sec. "Discussion"). Steps, for a parent n with children a, b:

  u_a = q_n o (P_b p_b)          (partial at the top of edge a)
  q_a = P_a^T u_a                (pre-order partial at the bottom of edge a)
  dlogL/dt_a = sum_p w_p [sum_r w_r u_a^T (dP_a/dt) p_a]
                         / [sum_r w_r u_a^T P_a p_a]

with q_root = pi in every category and dP/dt = rho Q P. The denominator is
the pattern likelihood up to the power-of-two scales of p and q, which
cancel in the ratio. Substitution parameters (Sec. "Discussion": exact
reverse-mode gradients through the matrix exponential) use the same ratio
with dP/dtheta = Frechet derivative of expm at rho t Q in direction
rho t dQ/dtheta.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm_frechet

from .pruning import (_rescale, child_product, derivative_matrices, post_order,
                      tip_partials, transition_matrices)


def pre_order(children: np.ndarray, n_tips: int, P: np.ndarray, post: dict,
              tips: np.ndarray, pi, R: int, rescale: bool = True):
    """Pre-order partials q[v] ([R, P, S]) and edge-top partials u[v] for
    every non-root node v, plus the per-node post-order child products."""
    children = np.asarray(children)
    root = 2 * n_tips - 2
    n_pat = tips.shape[1]
    S = P.shape[-1]

    def get(v):
        return tips[v] if v < n_tips else post[v]

    q = {root: np.broadcast_to(np.asarray(pi, float), (R, n_pat, S)).copy()}
    u = {}
    for n in range(root, n_tips - 1, -1):
        a, b = children[n - n_tips]
        va = child_product(P[a], get(a))
        vb = child_product(P[b], get(b))
        for c, sib in ((a, vb), (b, va)):
            u[c] = q[n] * sib
            qc = np.einsum("rji,rpj->rpi", P[c], u[c])
            if rescale:
                qc, _ = _rescale(qc)
            q[c] = qc
    return q, u


def _edge_ratio(u_c, M_c, P_c, p_c, cat_weights):
    """Per-pattern sum_r w_r u^T M p / sum_r w_r u^T P p."""
    num = np.einsum("r,rpi,rpi->p", cat_weights, u_c, child_product(M_c, p_c))
    den = np.einsum("r,rpi,rpi->p", cat_weights, u_c, child_product(P_c, p_c))
    return num / den


def branch_gradient(tree, Q, pi, rates, cat_weights, pattern_weights,
                    tip_states, rescale: bool = True, chunk: int = 8192):
    """dlogL/dt_v for every non-root node v (array of length 2N-1, root 0)."""
    S = Q.shape[0]
    n_tips = tree.n_tips
    R = len(rates)
    P = transition_matrices(Q, tree.edge_len, rates)
    dP = derivative_matrices(Q, P, rates)
    cw = np.asarray(cat_weights, float)
    w = np.asarray(pattern_weights, float)
    g = np.zeros(2 * n_tips - 1)
    for lo in range(0, tip_states.shape[1], chunk):
        tips = tip_partials(tip_states[:, lo:lo + chunk], S)
        post, _ = post_order(tree.children, n_tips, P, tips, rescale)
        _, u = pre_order(tree.children, n_tips, P, post, tips, pi, R, rescale)
        for v, uv in u.items():
            pv = tips[v] if v < n_tips else post[v]
            g[v] += np.dot(w[lo:lo + chunk], _edge_ratio(uv, dP[v], P[v], pv, cw))
    return g


def subst_gradient(tree, Q, dQs, pi, rates, cat_weights, pattern_weights,
                   tip_states, rescale: bool = True, chunk: int = 8192):
    """dlogL/dtheta for each dQ/dtheta in ``dQs`` (root frequencies fixed)."""
    S = Q.shape[0]
    n_tips = tree.n_tips
    rates = np.asarray(rates, float)
    R = len(rates)
    P = transition_matrices(Q, tree.edge_len, rates)
    dPs = []
    for dQ in dQs:
        d = np.empty_like(P)
        for v, t in enumerate(tree.edge_len):
            for r, rho in enumerate(rates):
                d[v, r] = expm_frechet(rho * t * Q, rho * t * dQ, compute_expm=False)
        dPs.append(d)
    cw = np.asarray(cat_weights, float)
    w = np.asarray(pattern_weights, float)
    g = np.zeros(len(dQs))
    for lo in range(0, tip_states.shape[1], chunk):
        tips = tip_partials(tip_states[:, lo:lo + chunk], S)
        post, _ = post_order(tree.children, n_tips, P, tips, rescale)
        _, u = pre_order(tree.children, n_tips, P, post, tips, pi, R, rescale)
        for v, uv in u.items():
            pv = tips[v] if v < n_tips else post[v]
            for k, d in enumerate(dPs):
                g[k] += np.dot(w[lo:lo + chunk], _edge_ratio(uv, d[v], P[v], pv, cw))
    return g


def edge_adjoints(tree, Q, pi, rates, cat_weights, pattern_weights, tip_states,
                  rescale: bool = True, chunk: int = 8192) -> np.ndarray:
    """M[v, r] = dlogL/dP_r(t_v) ([2N-2, R, S, S]) for every non-root node v.

    L_p is linear in each transition matrix (the pattern likelihood is
    sum_r w_r u_v^T P_v p_v for any edge v), so
      M[v, r] = w_r sum_p (w_p / L_p) u_v[r, p] p_v[r, p]^T,
    with L_p taken as that same-edge denominator (the power-of-two scales of
    u and p cancel in the ratio)."""
    S = Q.shape[0]
    n_tips = tree.n_tips
    R = len(rates)
    P = transition_matrices(Q, tree.edge_len, rates)
    cw = np.asarray(cat_weights, float)
    w = np.asarray(pattern_weights, float)
    M = np.zeros((2 * n_tips - 2, R, S, S))
    for lo in range(0, tip_states.shape[1], chunk):
        tips = tip_partials(tip_states[:, lo:lo + chunk], S)
        post, _ = post_order(tree.children, n_tips, P, tips, rescale)
        _, u = pre_order(tree.children, n_tips, P, post, tips, pi, R, rescale)
        for v, uv in u.items():
            pv = tips[v] if v < n_tips else post[v]
            den = np.einsum("r,rpi,rpi->p", cw, uv, child_product(P[v], pv))
            coef = w[lo:lo + chunk] / den
            pr = np.broadcast_to(pv, uv.shape)
            M[v] += np.einsum("r,p,rpi,rpj->rij", cw, coef, uv, pr)
    return M


def rate_matrix_gradient(tree, Q, pi, rates, cat_weights, pattern_weights, tip_states,
                         rescale: bool = True, first_order: bool = False,
                         chunk: int = 8192) -> np.ndarray:
    """dlogL/dQ ([S, S]): the derivative of logL with respect to every entry
    of Q, with P_r(t) = expm(rho_r t Q) and the root distribution pi fixed.

    By the chain rule, dlogL/dQ = sum_{v,r} of the adjoint of the Frechet
    derivative of expm at A = rho_r t_v Q applied to M[v, r] (edge_adjoints),
    scaled by rho_r t_v. For expm that adjoint is the Frechet derivative at
    A^T: <M, L(A, E)> = <L(A^T, M), E> (Sec. "Discussion": reverse-mode
    gradients through the adjoint of the matrix exponential).

    first_order: the approximation the paper describes for random-effects
    models (Sec. "Algorithmic advances"), dP ~ rho t dQ P, which gives
    sum_{v,r} rho_r t_v M[v, r] P_r(t_v)^T."""
    M = edge_adjoints(tree, Q, pi, rates, cat_weights, pattern_weights, tip_states,
                      rescale, chunk)
    rates = np.asarray(rates, float)
    S = Q.shape[0]
    G = np.zeros((S, S))
    for v, t in enumerate(tree.edge_len[: len(M)]):
        for r, rho in enumerate(rates):
            A = rho * t * Q
            if first_order:
                G += rho * t * M[v, r] @ expm_frechet(A, np.zeros_like(A))[0].T
            else:
                G += rho * t * expm_frechet(A.T, M[v, r], compute_expm=False)
    return G
