"""Node-height ratio transform on the device against the oracle: heights and
branch lengths exactly, and the chain rule from the GPU branch gradient to
ratios, root height and branch rates (FP64 and FP32 paths)."""
import numpy as np
import pytest

import synth
from oracle import gradient as og, model as om, ratio as orat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import build
    build.build()


def setup(n_tips=300, n_pat=2000, seed=3):
    w = synth.workload("gtr_512x100k", n_tips=n_tips, n_patterns=n_pat)
    rng = np.random.default_rng(seed)
    tip_h = rng.uniform(0.0, 0.2, n_tips)
    r = rng.uniform(0.3, 0.9, n_tips - 1)
    anc = orat.anchors(w.tree.children, n_tips, tip_h)
    root_h = anc[-1] + 0.8
    rate = rng.lognormal(0.0, 0.3, 2 * n_tips - 1)
    return w, tip_h, r, root_h, rate


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_ratio_transform_and_gradient(prec, tol):
    from paper_2606_27607_gb300 import TreeLikelihood
    from paper_2606_27607_gb300._lib import ratio_gradient, ratio_heights
    w, tip_h, r, root_h, rate = setup()
    N = w.tree.n_tips
    par = orat.parents(w.tree.children, N)
    h, t = ratio_heights(par, tip_h, r, root_h, rate)
    want_h = orat.heights(w.tree.children, N, tip_h, r, root_h)
    want_t = orat.branch_lengths(w.tree.children, N, want_h, rate)
    assert np.allclose(h, want_h, rtol=1e-15, atol=1e-15)
    assert np.allclose(t, want_t, rtol=1e-14, atol=1e-15)
    tl = TreeLikelihood(N, w.n_patterns, 4, 4, prec)
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, t)
        _, g = tl.gradient()
    finally:
        tl.close()
    gr, groot, grate = ratio_gradient(par, tip_h, r, root_h, rate, g)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    tree = synth.Tree(N, w.tree.children, w.tree.parent, want_t)
    wg = og.branch_gradient(tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    wr, wroot, wrate = orat.ratio_gradient(w.tree.children, N, tip_h, r, root_h, rate, wg)
    for got, want in ((gr[:-1], wr[:-1]), (grate[:-1], wrate[:-1])):
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * scale)) <= tol
    assert abs(groot - wroot) <= tol * max(abs(wroot), 1e-3 * np.max(np.abs(wr)))
    # the device chain rule on the GPU's own gradient equals the oracle's
    # chain rule on that same gradient to FP64 rounding
    er, eroot, erate = orat.ratio_gradient(w.tree.children, N, tip_h, r, root_h, rate, g)
    assert np.allclose(gr, er, rtol=1e-12, atol=1e-9 * np.max(np.abs(er)))
    assert np.allclose(grate, erate, rtol=1e-12, atol=1e-9 * np.max(np.abs(erate)))
