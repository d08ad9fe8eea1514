"""Codon (GY94, 61 states padded to 64) tensor-core path (tcgen05 kind::tf32)
against the FP64 oracle. Reduced-precision tolerance: 1e-5 relative on
logL. Per-pattern log-likelihoods: TF32 keeps 11 significant bits, so every
stored partial and every entry of P carries a relative rounding error up to
2^-11; a pattern accumulates about one such error per internal node, hence
|l_p - l_p*| <= 2^-11 * (N - 1)."""
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


def codon_workload(n_tips, n_patterns):
    return synth.workload("gy94_128x20k", n_tips=n_tips, n_patterns=n_patterns)


def run(w, prec, site=False, tips_as_partials=False):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 61, 4, prec)
    try:
        if tips_as_partials:
            for t in range(w.tree.n_tips):
                tl.inst.set_tip_partials(t, op.tip_partials(w.tips[t:t + 1], 61)[0])
        else:
            tl.set_tips(w.tips)
        tl.set_model("gy94", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        return tl.loglik(site=site)
    finally:
        tl.close()


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
@pytest.mark.parametrize("n_tips,n_pat", [(2, 1), (5, 150), (12, 300), (40, 257)])
def test_codon_tf32_matches_oracle(n_tips, n_pat, prec):
    w = codon_workload(n_tips, n_pat)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, want_site = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    logl, site = run(w, prec, site=True)
    assert abs(logl - want_l) <= 1e-5 * abs(want_l), (logl, want_l)
    assert np.max(np.abs(site - want_site)) <= 2.0 ** -11 * (n_tips - 1)


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
def test_codon_tf32_tip_states_equal_one_hot_partials_bit_exact(prec):
    w = codon_workload(9, 200)
    a = run(w, prec)
    b = run(w, prec, tips_as_partials=True)
    assert a == b


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
def test_codon_tf32_ambiguous_tips(prec):
    w = codon_workload(7, 130)
    rng = np.random.default_rng(3)
    w.tips = w.tips.copy()
    w.tips[rng.random(w.tips.shape) < 0.05] = 61
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    logl = run(w, prec)
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)


def test_codon_split_removes_the_shared_matrix_error():
    """A case where plain TF32 misses 1e-5 on logL (the matrices' rounding is
    common to every pattern and does not average out); with split matrices
    only the per-pattern rounding of stored partials remains."""
    import dataclasses

    import synth as sy
    chains, reqs, _ = sy.serving_stream(60, 8, taxa=(4, 40), patterns=(10, 3000))
    w0 = chains[6]
    assert w0.model == "gy94"
    errs = {"tf32": [], "tf32x2": []}
    for r in [r for r in reqs if r.chain == 6][:4]:
        tree = sy.Tree(w0.tree.n_tips, w0.tree.children, w0.tree.parent, r.edge_len)
        w = dataclasses.replace(w0, tree=tree, params=r.params)
        Q, pi, _ = om.build(w.model, w.params, w.freqs)
        want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
        for prec in errs:
            errs[prec].append(abs(run(w, prec) - want_l) / abs(want_l))
    assert max(errs["tf32x2"]) <= 1e-5, errs
    assert max(errs["tf32x2"]) < max(errs["tf32"]), errs


@pytest.mark.slow
def test_codon_128x20k_full_size_sampled():
    w = synth.workload("gy94_128x20k")
    logl, site = run(w, "tf32", site=True)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(w.n_patterns, 300, replace=False))
    idx[-1] = w.n_patterns - 1
    _, want_site = op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                     w.tips, patterns=idx)
    assert np.max(np.abs(site[idx] - want_site)) <= 2.0 ** -11 * 127
    assert abs(logl - np.sum(site)) <= 1e-9 * abs(logl)
    # the FP64 generic GPU path (itself oracle-checked at small sizes) agrees
    l64 = run(w, "f64")
    assert abs(logl - l64) <= 1e-5 * abs(l64)


def assert_grad_close(g, want, tol):
    scale = np.max(np.abs(want))
    den = np.maximum(np.abs(want), 1e-3 * scale)
    err = np.abs(g - want) / den
    assert np.max(err) <= tol, (np.max(err), int(np.argmax(err)))


@pytest.mark.parametrize("n_tips,n_pat", [(3, 40), (8, 150), (20, 300)])
def test_codon_tf32x2_gradient(n_tips, n_pat):
    """Split matrices: logL within 1e-5, gradient within 1e-3 in the 2-norm
    and every component within 1e-3 of the largest. The stored partials keep
    TF32's 11 bits, so a component whose per-pattern terms cancel to a small
    sum keeps an absolute error of order 2^-11 sqrt(P) of its terms."""
    from oracle import gradient as og
    from paper_2606_27607_gb300 import TreeLikelihood
    w = codon_workload(n_tips, n_pat)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    want_g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = TreeLikelihood(n_tips, n_pat, 61, 4, "tf32x2")
    try:
        tl.set_tips(w.tips)
        tl.set_model("gy94", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        logl, g = tl.gradient()
    finally:
        tl.close()
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)
    gv, wv = g[:-1], want_g[:-1]
    assert np.linalg.norm(gv - wv) <= 1e-3 * np.linalg.norm(wv)
    assert np.max(np.abs(gv - wv)) <= 1e-3 * np.max(np.abs(wv))


@pytest.mark.parametrize("n_tips,n_pat", [(3, 40), (8, 150), (20, 300)])
def test_codon_tf32_gradient_matches_oracle(n_tips, n_pat):
    from oracle import gradient as og
    from paper_2606_27607_gb300 import TreeLikelihood
    w = codon_workload(n_tips, n_pat)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    want_g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = TreeLikelihood(n_tips, n_pat, 61, 4, "tf32")
    try:
        tl.set_tips(w.tips)
        tl.set_model("gy94", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        logl, g = tl.gradient()
    finally:
        tl.close()
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)
    # plain TF32 (11-bit operands): relative error of the gradient vector, and
    # each component within 1e-3 of the largest; components whose per-pattern
    # terms cancel need the split mode for the per-component bound
    gv, wv = g[:-1], want_g[:-1]
    assert np.linalg.norm(gv - wv) <= 1e-3 * np.linalg.norm(wv)
    assert np.max(np.abs(gv - wv)) <= 1e-3 * np.max(np.abs(wv))
