"""Degenerate and boundary inputs against the FP64 oracle: zero-length and
very long branches, patterns whose tips are all ambiguous, two taxa,
non-uniform pattern weights with a zero weight, codon instances with fewer
than four categories, batched instances with three categories, and an op
list that covers part of the tree."""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import gradient as og, model as om, pruning as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import build
    build.build()


def want(w, grad=True):
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    logl, site = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    g = (og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
         if grad else None)
    return logl, site, g


def got(w, prec, grad=True):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, len(w.rates), prec)
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        if grad:
            logl, g = tl.gradient()
            return logl, None, g
        logl, site = tl.loglik(site=True)
        return logl, site, None
    finally:
        tl.close()


TOL = {"f64": (1e-11, 1e-10), "f32": (1e-5, 1e-3), "tf32x2": (1e-5, None), "tf32x3": (1e-5, 1e-3)}


def check(w, prec, grad=True):
    wl, _, wg = want(w, grad)
    gl, _, gg = got(w, prec, grad)
    tl_, tg = TOL[prec]
    assert abs(gl - wl) <= tl_ * abs(wl), (gl, wl)
    if grad:
        assert tg is not None, f"{prec} is a log-likelihood mode"
        scale = np.max(np.abs(wg))
        err = np.abs(gg - wg) / np.maximum(np.abs(wg), 1e-3 * scale)
        assert np.max(err) <= tg, (np.max(err), int(np.argmax(err)))


def nuc(n_tips=17, n_pat=300):
    return synth.workload("gtr_512x100k", n_tips=n_tips, n_patterns=n_pat)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_zero_and_very_long_branches(prec):
    """t = 0 (P = I, dP/dt = rho Q) on one tip edge and one internal edge;
    t = 40 (P near 1 pi^T) on another."""
    w = nuc()
    el = w.tree.edge_len.copy()
    el[0] = 0.0
    el[w.tree.n_tips + 2] = 0.0
    el[3] = 40.0
    w = dataclasses.replace(w, tree=synth.Tree(w.tree.n_tips, w.tree.children, w.tree.parent, el))
    check(w, prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_all_ambiguous_patterns_and_weights(prec):
    """Patterns whose tips are all ambiguous have likelihood 1 (site logL 0);
    weights 0, 1 and 5."""
    w = nuc(n_pat=257)
    tips = w.tips.copy()
    tips[:, :7] = 4           # any code outside 0..3 is ambiguous
    tips[:5, 200] = -1
    wt = np.ones(w.n_patterns)
    wt[10] = 0.0
    wt[11:20] = 5.0
    w = dataclasses.replace(w, tips=tips, pattern_weights=wt)
    check(w, prec)
    _, site, _ = got(w, prec, grad=False)
    assert np.all(np.abs(site[:7]) <= (1e-12 if prec == "f64" else 1e-6))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_two_taxa(prec):
    check(nuc(n_tips=2, n_pat=130), prec)


@pytest.mark.parametrize("ncat", [1, 2, 3])
def test_codon_fewer_categories(ncat):
    """The tensor-core kernels with R < 4 (TMEM columns of absent
    categories unused)."""
    w = synth.workload("gy94_128x20k", n_tips=7, n_patterns=150)
    rates = synth.gamma_rates(0.5, ncat)
    w = dataclasses.replace(w, rates=rates, cat_weights=np.full(ncat, 1.0 / ncat))
    check(w, "tf32x3")
    check(w, "tf32x2", grad=False)


def test_batched_three_categories():
    import torch
    from paper_2606_27607_gb300 import TreeLikelihood
    from paper_2606_27607_gb300._lib import Batch
    ws = [nuc(n_tips=n, n_pat=p) for n, p in ((9, 100), (30, 333), (4, 65))]
    ws = [dataclasses.replace(w, rates=synth.gamma_rates(0.5, 3), cat_weights=np.full(3, 1 / 3))
          for w in ws]
    tls = []
    for w in ws:
        tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 3, "f32")
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        tl.update_matrices(True)
        tls.append(tl)
    b = Batch()
    try:
        b.update_partials([t.inst for t in tls], [t._post for t in tls])
        out = torch.zeros(len(tls), dtype=torch.float64, device="cuda")
        b.root_loglik_dev([t.inst for t in tls], [t.nn - 1 for t in tls], [0] * 3, out.data_ptr())
        gs = [torch.zeros(t.nn, dtype=torch.float64, device="cuda") for t in tls]
        b.pre_order_gradient_dev([t.inst for t in tls], [t._pre for t in tls], [0] * 3,
                                 [g.data_ptr() for g in gs], [t.nn for t in tls])
        torch.cuda.synchronize()
        for k, w in enumerate(ws):
            wl, _, wg = want(w)
            assert abs(float(out[k]) - wl) <= 1e-5 * abs(wl)
            g = gs[k].cpu().numpy()
            scale = np.max(np.abs(wg))
            assert np.max(np.abs(g - wg) / np.maximum(np.abs(wg), 1e-3 * scale)) <= 1e-3
    finally:
        b.close()
        for t in tls:
            t.close()


def test_partial_traversal_of_a_subtree():
    """An op list for one subtree only: its root's partial equals the
    oracle's post-order partial of that node (same rescaling)."""
    from paper_2606_27607_gb300 import TreeLikelihood
    w = nuc(n_tips=12, n_pat=200)
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, "f64")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        tl.update_matrices(False)
        ops = tl._post
        node = w.tree.n_tips + 4     # an internal node and the ops below it
        keep = []
        below = {node}
        for o in reversed(ops):
            if o["dest"] in below:
                keep.append(o)
                for c in (o["child1"], o["child2"]):
                    if c >= w.tree.n_tips:
                        below.add(c)
        sub = np.array(list(reversed(keep)), dtype=ops.dtype)
        tl.inst.update_partials(sub)
        part, expo = tl.inst.get_partials(node)
    finally:
        tl.close()
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    P = op.transition_matrices(Q, w.tree.edge_len, w.rates)
    tips = op.tip_partials(w.tips, 4)
    post, scales = op.post_order(w.tree.children, w.tree.n_tips, P, tips, True)

    def cum(v):  # exponents removed in v's subtree (the oracle records each node's own)
        if v < w.tree.n_tips:
            return 0
        a, b = w.tree.children[v - w.tree.n_tips]
        return scales[v] + cum(a) + cum(b)

    want_p = post[node] * np.exp2(cum(node))[None, :, None]
    got_p = part * np.exp2(expo)[None, :, None]
    assert np.allclose(got_p, want_p, rtol=1e-11, atol=0)
