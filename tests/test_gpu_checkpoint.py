"""Subtree checkpointing: logL and every branch derivative with post-order
partials kept only at checkpoint depths (the rest recomputed in the
pre-order pass) are bit-identical to the whole-tree pass, in fewer
buffers."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import build
    build.build()


def whole(w, prec):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, 4, prec)
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        return tl.gradient()
    finally:
        tl.close()


@pytest.mark.parametrize("name,prec,kw", [("gtr_512x100k", "f32", dict(n_tips=200, n_patterns=3000)),
                                          ("gtr_512x100k", "f64", dict(n_tips=90, n_patterns=500)),
                                          ("gy94_64x5k", "tf32x2", dict(n_tips=40, n_patterns=300)),
                                          ("gy94_64x5k", "tf32x3", dict(n_tips=40, n_patterns=300)),
                                          ("gy94_64x5k", "f64", dict(n_tips=12, n_patterns=100))])
@pytest.mark.parametrize("band", [1, 2, 3, 5])
def test_checkpointed_gradient_is_bit_identical(name, prec, kw, band):
    from paper_2606_27607_gb300.checkpoint import CheckpointedLikelihood
    w = synth.workload(name, **kw)
    want_l, want_g = whole(w, prec)
    ck = CheckpointedLikelihood(w.tree.n_tips, w.n_patterns, w.tree.children, w.n_states, 4,
                                prec, band=band)
    try:
        ck.set_data(w.tips, w.model, w.params, w.freqs, w.rates, w.cat_weights)
        logl, g = ck.gradient(w.tree.edge_len)
        nbuf = ck.n_buffers
    finally:
        ck.close()
    assert logl == want_l
    assert np.array_equal(g, want_g)
    if band >= 2 and w.tree.n_tips >= 90:
        assert nbuf < 0.75 * 2 * (w.tree.n_tips - 1)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_pattern_chunks_sum_to_the_whole(prec, tol):
    """Patterns in consecutive blocks on one instance sized for a block:
    logL and gradient equal the whole-alignment evaluation up to the order
    of the pattern sums."""
    from paper_2606_27607_gb300.shard import ChunkedLikelihood
    w = synth.workload("gtr_512x100k", n_tips=60, n_patterns=5003)
    want_l, want_g = whole(w, prec)
    ch = ChunkedLikelihood(w.tree.n_tips, w.n_patterns, 3, 4, 4, prec)
    try:
        ch.set_data(w.tips, w.model, w.params, w.freqs, w.rates, w.cat_weights)
        logl, g = ch.gradient(w.tree.children, w.tree.edge_len)
    finally:
        ch.close()
    assert abs(logl - want_l) <= tol * abs(want_l)
    assert np.max(np.abs(g - want_g)) <= tol * np.max(np.abs(want_g))
