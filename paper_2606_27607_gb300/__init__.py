"""treelik: GB300-native (sm_103a) phylogenetic log-likelihood and gradient.

The C ABI (include/treelik.h, libtreelik.so) does all device work; this
package only marshals arguments (``_lib``), builds operation lists from a
tree (``tree``) and bundles the calls one likelihood or gradient evaluation
makes (``TreeLikelihood``).
"""
from __future__ import annotations

import numpy as np

from . import tree as _tree
from ._lib import (EDGE_DTYPE, OP_DTYPE, PRE_OP_DTYPE, Instance, TreelikError,  # noqa: F401
                   load)

__all__ = ["Instance", "TreeLikelihood", "TreelikError", "load", "LogLikelihood"]


class TreeLikelihood:
    """One tree, one model slot, resident on the device.

    Node v (tips 0..N-1, internal N..2N-2 in post-order, root 2N-2) uses
    buffer v for its post-order partials; the edge above v uses matrix slot v
    for P and n_nodes + v for dP/dt. Pre-order partials of internal node v
    live in buffer pre_base + v.
    """

    def __init__(self, n_tips: int, n_patterns: int, n_states: int = 4, n_categories: int = 4,
                 precision: str = "f32", stream: int | None = None, store_pre: bool = False,
                 scale: bool = True):
        N = n_tips
        self.N, self.P, self.S, self.R = N, n_patterns, n_states, n_categories
        self.nn = 2 * N - 1
        # q of node v lives in buffer pre_base + v (internal nodes only unless
        # store_pre, which also keeps the tips' q for tl_edge_derivatives)
        self.pre_base = (2 * N - 1) if store_pre else (N - 1)
        self.store_pre = store_pre
        n_buffers = (N - 1) + (self.nn if store_pre else N - 1)
        self.inst = Instance(N, n_patterns, n_states, n_categories, n_buffers, 2 * self.nn, 1,
                             precision, scale, stream)
        self.children = None
        self._post = None
        self._pre = None
        # bumped by every call that changes the device state an adjoint
        # reads (inputs, model, tree, post-order partials), so a caller that
        # saved the state of one evaluation can tell whether it is current
        self.generation = 0

    def _touch(self) -> None:
        self.generation += 1

    def close(self):
        self.inst.close()

    # inputs ----------------------------------------------------------------
    def set_tips(self, tips: np.ndarray) -> None:
        self._touch()
        for t in range(self.N):
            self.inst.set_tip_states(t, tips[t])

    N_PARAMS = {"hky": 1, "gtr": 6, "gy94": 2, "gy94re": 265}

    def set_model(self, kind: str, params, freqs) -> None:
        self._touch()
        self.inst.set_model(0, kind, params, freqs)
        self.kind = kind

    def set_rates(self, rates, weights=None) -> None:
        self._touch()
        self.inst.set_category_rates(rates)
        if weights is not None:
            self.inst.set_category_weights(weights)

    def set_pattern_weights(self, w) -> None:
        self._touch()
        self.inst.set_pattern_weights(w)

    def set_tree(self, children, edge_len) -> None:
        self._touch()
        children = np.asarray(children)
        if self.children is None or not np.array_equal(children, self.children):
            self.children = children.copy()
            self._post = _tree.post_ops(children, self.N)
            self._pre = _tree.pre_ops(children, self.N, self.pre_base)
            self._preq = _tree.q_ops(children, self.N, self.pre_base)
            self._adj = _tree.adj_ops(children, self.N, self.pre_base)
        self.edge_len = np.asarray(edge_len, dtype=np.float64)

    # evaluation ------------------------------------------------------------
    def update_matrices(self, derivatives: bool) -> None:
        v = np.arange(self.nn - 1, dtype=np.int32)   # every non-root node
        dp = (self.nn + v).astype(np.int32) if derivatives else None
        self.inst.update_matrices(0, v, self.edge_len[: self.nn - 1], dp)

    def loglik(self, site: bool = False, derivatives: bool = False):
        """logL (and per-pattern values); ``derivatives`` also fills the
        dP/dt slots so that branch_gradient() can follow without a second
        post-order pass."""
        self._touch()
        self.update_matrices(derivatives)
        self.inst.update_partials(self._post)
        return self.inst.root_loglik(self.nn - 1, 0, site)

    def branch_gradient(self) -> np.ndarray:
        """dlogL/dt for every node (root entry 0) from the post-order
        partials and dP/dt of the last loglik(derivatives=True)."""
        return self.inst.pre_order_gradient(self._pre, self.nn, 0)

    def gradient(self):
        """(logL, dlogL/dt for every node, root entry 0)."""
        self._touch()
        self.update_matrices(True)
        self.inst.update_partials(self._post)
        logl = self.inst.root_loglik(self.nn - 1, 0)
        g = self.inst.pre_order_gradient(self._pre, self.nn, 0)
        return logl, g

    def subst_gradient(self) -> np.ndarray:
        """dlogL/dtheta for every parameter of the model (kappa for HKY, the
        six exchangeabilities for GTR, kappa and omega for GY94), with the
        post-order partials of the current tree. One pre-order pass per
        parameter with dP/dtheta in the derivative slots; the next gradient()
        recomputes dP/dt there."""
        self._touch()   # the derivative slots now hold dP/dtheta
        n = len(self.inst.get_model(0)[2])   # the model's dQ/dtheta matrices
        v = np.arange(self.nn - 1, dtype=np.int32)
        out = np.zeros(n)
        for k in range(n):
            self.inst.update_param_matrices(0, k, self.nn + v, self.edge_len[: self.nn - 1])
            out[k] = self.inst.pre_order_derivative(self._pre, self.nn, 0).sum()
        return out

    def adjoint(self, first_order: bool = False):
        """Reverse-mode gradient after loglik(): one pre-order pass storing q,
        then one pass over the partials (tl_adjoint). Returns (dlogL/dt per
        node (root 0), dlogL/dQ [S, S], dlogL/dtheta). ``first_order`` takes
        dlogL/dQ by the approximation dP = rho t dQ P."""
        self.inst.update_pre_partials(self._preq, 0)
        return self.inst.adjoint(self._adj, self.nn, self.n_params(), 0, first_order)

    def n_params(self) -> int:
        """Parameters of the current model (S x S exchangeabilities for the
        general reversible model)."""
        kind = getattr(self, "kind", None)
        return self.S * self.S if kind == "rev" else self.N_PARAMS.get(kind, 0)

    def value_and_grad(self):
        """(logL, dlogL/dt per node, dlogL/dtheta) in one forward/backward."""
        logl = self.loglik()
        g, _, th = self.adjoint()
        return logl, g, th


def __getattr__(name):
    if name == "LogLikelihood":
        from .autograd import LogLikelihood
        return LogLikelihood
    raise AttributeError(name)
