"""A pattern whose likelihood underflows in FP32 storage: one subtree that
needs many substitutions (only the fastest rate category survives the
shared per-pattern scale) joined to one that needs none over long branches
(only the slowest survives), so the parent's product is zero in every
category. The FP64 path and the oracle agree on the value; the TF32 path
reports TL_ERR_NUMERIC; the server re-evaluates such a request in FP64."""
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


def crafted():
    n = 64
    children, edge = [], np.zeros(2 * n - 1)
    # at the root the largest product per category is about 1e-72, 1e-50,
    # 1e-56 and 1e-114 (oracle): below the smallest FP32 value in every one
    ra, nxt = balanced(range(32), n, children, edge, 0.003)
    rb, nxt = balanced(range(32, 64), nxt, children, edge, 5.0)
    children.append((ra, rb))
    edge[ra], edge[rb] = 0.003, 5.0
    children = np.array(children)
    parent = -np.ones(2 * n - 1, dtype=np.int64)
    for k, (a, b) in enumerate(children):
        parent[a] = parent[b] = n + k
    tree = synth.Tree(n, children, parent, edge)
    tips = np.zeros((n, 2), dtype=np.int8)
    tips[:32, 0] = np.arange(0, 64, 2)[:32] % 61     # 32 different codons, short branches
    tips[32:, 0] = 7                                  # one codon, long branches
    tips[:, 1] = 7                                    # an ordinary pattern
    w = synth.workload("gy94_64x5k", n_tips=n, n_patterns=2)
    return dataclasses.replace(w, tree=tree, tips=tips)


def test_fp32_underflow_is_reported_and_fp64_is_exact():
    from paper_2606_27607_gb300 import TreeLikelihood, TreelikError
    w = crafted()
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)[0]
    res = {}
    for prec in ("f64", "tf32x2"):
        tl = TreeLikelihood(64, 2, 61, 4, prec)
        try:
            tl.set_tips(w.tips)
            tl.set_model(w.model, w.params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            try:
                res[prec] = tl.loglik()
            except TreelikError as e:
                res[prec] = e
        finally:
            tl.close()
    assert abs(res["f64"] - want) <= 1e-11 * abs(want)
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
    tl = TreeLikelihood(64, 2, 61, 4, "f64")
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
    whole = footprint(64, 2, 61, "tf32x3")
    band, nb = best_band(w.tree.children, 64)
    budget = (whole + footprint(64, 2, 61, "tf32x3", nb)) // 2
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
    assert abs(got.logl - want) <= 1e-11 * abs(want)
    assert got.gradient is not None and np.all(np.isfinite(got.gradient))
