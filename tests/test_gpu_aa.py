"""Twenty states (amino acids under a general reversible model): the split
tensor-core path with states padded to 64 and the FP64 generic path,
against the oracle: logL, branch gradients, dlogL/dQ and the gradient with
respect to every exchangeability (complex-step dQ/dE in the oracle), every
component within |x - x*| <= tol max(|x*|, 1e-3 |x*|_inf)."""
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


@pytest.mark.parametrize("prec,tol_l,tol_g", [("f64", 1e-11, 1e-10), ("tf32x3", 1e-5, 1e-3)])
def test_amino_acid_loglik_gradient_and_adjoint(prec, tol_l, tol_g):
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload("aa20_256x10k", n_tips=9, n_patterns=333)
    tips = w.tips.copy()
    tips[0, :5] = 25          # ambiguous codes
    Q, pi, _ = om.build("rev", w.params, w.freqs)
    args = (w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, tips)
    want_l = op.loglik(*args)[0]
    want_g = og.branch_gradient(*args)
    want_q = og.rate_matrix_gradient(*args)
    want_th = np.einsum("kij,ij->k", om.rate_jacobian("rev", w.params, w.freqs), want_q)
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 20, 4, prec)
    try:
        tl.set_tips(tips)
        tl.set_model("rev", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        logl, g = tl.gradient()
        tl.loglik()
        g2, dq, th = tl.adjoint()
    finally:
        tl.close()
    assert abs(logl - want_l) <= tol_l * abs(want_l)
    assert th.size == 400           # the exchangeability matrix, diagonal 0
    assert np.all(th.reshape(20, 20).diagonal() == 0)
    for got, want in ((g[:-1], want_g[:-1]), (g2[:-1], want_g[:-1]), (dq, want_q), (th, want_th)):
        scale = np.max(np.abs(want))
        assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * scale)) <= tol_g
