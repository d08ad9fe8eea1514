"""Post-order pruning with transition matrices formed on the fly from the
eigensystem (one or a few site patterns, large state spaces) against the
oracle (expm) and against the stored-matrix path of the same instance."""
import dataclasses

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


CASES = [("aa20_256x10k", dict(n_tips=64, n_patterns=1)),
         ("gy94_64x5k", dict(n_tips=40, n_patterns=1)),
         ("gy94_64x5k", dict(n_tips=17, n_patterns=3)),
         ("gtr_512x100k", dict(n_tips=33, n_patterns=70))]


@pytest.mark.parametrize("name,kw", CASES)
def test_on_the_fly_matches_oracle_and_stored_matrices(name, kw):
    from paper_2606_27607_gb300 import TreeLikelihood, tree
    w = synth.workload(name, **kw)
    tips = w.tips.copy()
    tips[1, 0] = 99                     # an ambiguous code
    w = dataclasses.replace(w, tips=tips)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)[0]
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, "f64")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        stored = tl.loglik()
        tl.inst.update_partials_eigen(tree.eig_ops(w.tree.children, w.tree.n_tips,
                                                   w.tree.edge_len))
        fly = tl.inst.root_loglik(tl.nn - 1, 0)
    finally:
        tl.close()
    assert abs(fly - want) <= 1e-11 * abs(want), (fly, want)
    assert abs(fly - stored) <= 1e-12 * abs(stored)


def test_on_the_fly_rejects_bad_order_and_precision():
    from paper_2606_27607_gb300 import TreeLikelihood, TreelikError, tree
    w = synth.workload("aa20_256x10k", n_tips=6, n_patterns=1)
    tl = TreeLikelihood(6, 1, 20, 4, "f64")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        ops = tree.eig_ops(w.tree.children, 6, w.tree.edge_len)
        with pytest.raises(TreelikError, match="TL_ERR_ORDER|TL_ERR_STATE"):
            tl.inst.update_partials_eigen(ops[::-1].copy())   # parents before children
    finally:
        tl.close()
    tl = TreeLikelihood(6, 1, 20, 4, "tf32")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        with pytest.raises(TreelikError, match="TL_ERR_UNSUPPORTED"):
            tl.inst.update_partials_eigen(tree.eig_ops(w.tree.children, 6, w.tree.edge_len))
    finally:
        tl.close()
