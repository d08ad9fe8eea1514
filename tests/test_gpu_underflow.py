"""Patterns near and past the FP32 range: one subtree that needs many
substitutions (only the fastest rate categories survive the shared
per-pattern scale) joined to one that needs none over long branches (only
the slowest survive), so the root's product of the two children is tiny in
every category.

With 32 tips per subtree the largest normalised product is about 2^-165
(oracle): the TF32 path keeps it, since its stored partials carry a
per-pattern maximum near 2^48 and two children's product gains 2^96 of
headroom, and its logL and gradient match the oracle. With 64 tips per
subtree it is 2^-347, below FP32 with any headroom: the FP64 path and the
oracle agree, the TF32 path reports TL_ERR_NUMERIC and the server
re-evaluates such a request in FP64."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import model as om, pruning as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import build
    build.build()


# The FP64 path forms P from the eigensystem of Q, whose error is absolute in
# each entry (about 1e-16 times the conditioning of the eigenvectors, which
# grows as 1/sqrt(pi_min) for F3x4 frequencies); pattern 0's likelihood is a
# product of short-branch probabilities between distinct codons, entries far
# below 1, so that absolute error becomes a relative error of its logL near
# 1e-9 for 128 taxa (the oracle's P uses scaling and squaring instead).
F64_TOL = 1e-8


def balanced(tips, nxt, children, edge, t):
    """Join the given nodes pairwise into a balanced subtree, labels from nxt."""
    level = list(tips)
    while len(level) > 1:
        up = []
        for i in range(0, len(level), 2):
            a, b = level[i], level[i + 1]
            children.append((a, b))
            edge[a], edge[b] = t, t
            up.append(nxt)
            nxt += 1
        level = up
    return level[0], nxt


def crafted(n=128):
    """Two balanced subtrees of n/2 tips joined at the root. Largest
    normalised product of the root's children per category (oracle), pattern
    0: n = 64: 2^-239, 2^-165, 2^-185, 2^-378; n = 128: 2^-516, 2^-347,
    2^-376, 2^-756."""
    h = n // 2
    children, edge = [], np.zeros(2 * n - 1)
    ra, nxt = balanced(range(h), n, children, edge, 0.003)
    rb, nxt = balanced(range(h, n), nxt, children, edge, 5.0)
    children.append((ra, rb))
    edge[ra], edge[rb] = 0.003, 5.0
    children = np.array(children)
    parent = -np.ones(2 * n - 1, dtype=np.int64)
    for k, (a, b) in enumerate(children):
        parent[a] = parent[b] = n + k
    tree = synth.Tree(n, children, parent, edge)
    tips = np.zeros((n, 2), dtype=np.int8)
    tips[:h, 0] = np.arange(0, 2 * h, 2)[:h] % 61    # different codons, short branches
    tips[h:, 0] = 7                                  # one codon, long branches
    tips[:, 1] = 7                                   # an ordinary pattern
    w = synth.workload("gy94_64x5k", n_tips=n, n_patterns=2)
    return dataclasses.replace(w, tree=tree, tips=tips)


def evaluate(w, prec, gradient=False):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, 2, 61, 4, prec)
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        return tl.gradient() if gradient else tl.loglik()
    finally:
        tl.close()


@pytest.mark.parametrize("prec", ["tf32", "tf32x2", "tf32x3"])
def test_near_underflow_pattern_kept_by_tf32_headroom(prec):
    from oracle import gradient as og
    w = crafted(64)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)[0]
    want_g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                w.tips)
    logl, g = evaluate(w, prec, gradient=True)
    if prec == "tf32":
        # TF32 matrices and partials: L_p is multilinear in the matrices with
        # non-negative terms, so rounding each matrix and each stored partial
        # to TF32 (unit roundoff 2^-11) moves log L_p by at most
        # (edges + internal nodes) 2^-11 to first order
        n = w.tree.n_tips
        tol = w.tips.shape[1] * ((2 * n - 2) + (n - 1)) * 2.0 ** -11
    else:
        tol = 1e-5 * abs(want)
    assert abs(logl - want) <= tol
    assert np.all(np.isfinite(g))
    if prec == "tf32x3":   # the precision whose gradients meet the per-component bound
        g, want_g = np.asarray(g)[:-1], np.asarray(want_g)[:-1]
        scale = np.max(np.abs(want_g))
        err = np.abs(g - want_g) / np.maximum(np.abs(want_g), 1e-3 * scale)
        assert err.max() <= 1e-3, err.max()


def test_fp32_underflow_is_reported_and_fp64_is_exact():
    from paper_2606_27607_gb300 import TreelikError
    w = crafted()
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)[0]
    res = {}
    for prec in ("f64", "tf32x2"):
        try:
            res[prec] = evaluate(w, prec)
        except TreelikError as e:
            res[prec] = e
    assert abs(res["f64"] - want) <= F64_TOL * abs(want)
    assert isinstance(res["tf32x2"], TreelikError) and "TL_ERR_NUMERIC" in str(res["tf32x2"])


def test_server_falls_back_to_fp64():
    from paper_2606_27607_gb300 import TreeLikelihood
    from paper_2606_27607_gb300.serve import Server
    w = crafted()
    req = synth.ServingRequest(chain=0, edge_len=w.tree.edge_len, params=np.asarray(w.params),
                               gradient=True)
    s = Server()
    try:
        s.add_chain(w)
        f = s.submit(req)
        s.drain()
        got = f.result()
        stats = dict(s.stats)
    finally:
        s.close()
    tl = TreeLikelihood(w.tree.n_tips, 2, 61, 4, "f64")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        want_l, want_g = tl.gradient()
    finally:
        tl.close()
    assert stats.get("fp64_fallback", 0) == 1
    assert got.logl == want_l
    assert np.array_equal(got.gradient, want_g)


def test_server_falls_back_to_fp64_on_a_checkpointed_chain():
    """The same pattern on a chain whose whole-tree buffers exceed the
    budget: served with checkpointing, re-evaluated in FP64 in that form."""
    from paper_2606_27607_gb300.checkpoint import best_band
    from paper_2606_27607_gb300.serve import Server, footprint
    w = crafted()
    n = w.tree.n_tips
    whole = footprint(n, 2, 61, "tf32x3")
    band, nb = best_band(w.tree.children, n)
    budget = (whole + footprint(n, 2, 61, "tf32x3", nb)) // 2
    req = synth.ServingRequest(chain=0, edge_len=w.tree.edge_len, params=np.asarray(w.params),
                               gradient=True)
    s = Server(memory_budget=budget)
    try:
        s.add_chain(w)
        f = s.submit(req)
        s.drain()
        got = f.result()
        stats = dict(s.stats)
    finally:
        s.close()
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)[0]
    assert stats.get("checkpointed", 0) == 1 and stats.get("fp64_fallback", 0) == 1
    assert abs(got.logl - want) <= F64_TOL * abs(want)
    assert got.gradient is not None and np.all(np.isfinite(got.gradient))
