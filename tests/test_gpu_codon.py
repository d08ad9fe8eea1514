"""Codon (GY94, 61 states padded to 64) tensor-core path (tcgen05 kind::tf32)
against the FP64 oracle. Reduced-precision tolerance: 1e-5 relative on
logL, and per gradient component |g - g*| <= 1e-3 max(|g*|, 1e-3 |g*|_inf).
Per-pattern log-likelihoods: TF32 keeps 11 significant bits, so with
TF32-stored partials (tf32, tf32x2) every stored partial carries a relative
rounding error up to 2^-11; a pattern accumulates about one such error per
internal node, hence |l_p - l_p*| <= 2^-11 * (N - 1). Those two modes are
logL modes: a gradient component whose per-pattern terms cancel keeps an
absolute error of order 2^-11 sqrt(P) of its terms. tf32x3 stores FP32
partials and splits them on chip (three products, about 21 bits of both
operands): |l_p - l_p*| <= 2^-20 * (N - 1), and gradients meet the
per-component bound."""
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


SITE_BITS = {"tf32": 11, "tf32x2": 11, "tf32x3": 20}


@pytest.mark.parametrize("prec", ["tf32", "tf32x2", "tf32x3"])
@pytest.mark.parametrize("n_tips,n_pat", [(2, 1), (5, 150), (12, 300), (40, 257)])
def test_codon_tf32_matches_oracle(n_tips, n_pat, prec):
    w = codon_workload(n_tips, n_pat)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, want_site = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    logl, site = run(w, prec, site=True)
    assert abs(logl - want_l) <= 1e-5 * abs(want_l), (logl, want_l)
    assert np.max(np.abs(site - want_site)) <= 2.0 ** -SITE_BITS[prec] * max(n_tips - 1, 1)


@pytest.mark.parametrize("prec", ["tf32", "tf32x2", "tf32x3"])
def test_codon_degenerate_spectrum_matches_oracle(prec):
    """Uniform codon frequencies with kappa = omega = 1: the rate matrix has
    many repeated eigenvalues, which the eigensystem's refinement leaves to
    its FP64 Jacobi sweeps. Per-pattern bounds as above; the 1e-5 logL bound
    for the FP32-stored mode. With TF32-stored partials the logL is held to
    the sum of the per-pattern bounds: the symmetric model makes many
    partial entries equal, so their TF32 rounding errors do not cancel
    (tf32x2 measured 1.2e-5 relative here)."""
    import dataclasses
    w = codon_workload(12, 300)
    w = dataclasses.replace(w, params=np.array([1.0, 1.0]), freqs=np.full((3, 4), 0.25))
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, want_site = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    logl, site = run(w, prec, site=True)
    site_tol = 2.0 ** -SITE_BITS[prec] * 11
    assert np.max(np.abs(site - want_site)) <= site_tol
    if prec == "tf32x3":
        assert abs(logl - want_l) <= 1e-5 * abs(want_l), (logl, want_l)
    else:
        assert abs(logl - want_l) <= site_tol * np.sum(w.pattern_weights), (logl, want_l)


@pytest.mark.parametrize("prec", ["tf32", "tf32x2", "tf32x3"])
def test_codon_tf32_tip_states_equal_one_hot_partials_bit_exact(prec):
    w = codon_workload(9, 200)
    a = run(w, prec)
    b = run(w, prec, tips_as_partials=True)
    assert a == b


@pytest.mark.parametrize("prec", ["tf32", "tf32x2", "tf32x3"])
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


@pytest.mark.parametrize("n_tips,n_pat", [(3, 40), (8, 150), (20, 300), (7, 161)])
def test_codon_tf32x3_gradient_matches_oracle(n_tips, n_pat):
    """Split partials and matrices: logL within 1e-5 and every branch
    derivative within the per-component bound (the fused pre-order pass and
    the reverse-mode adjoint)."""
    from oracle import gradient as og
    from paper_2606_27607_gb300 import TreeLikelihood
    w = codon_workload(n_tips, n_pat)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    want_g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = TreeLikelihood(n_tips, n_pat, 61, 4, "tf32x3")
    try:
        tl.set_tips(w.tips)
        tl.set_model("gy94", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        logl, g = tl.gradient()
        tl.loglik()
        g2, _, _ = tl.adjoint()
    finally:
        tl.close()
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-3)
    assert_grad_close(g2[:-1], want_g[:-1], 1e-3)


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
def test_fused_post_order_is_bit_identical_to_level_kernels(prec, monkeypatch):
    """The subtree-fused post-order kernel (one CTA walks the whole op list
    for a pattern tile, each op's result kept in tensor memory as the next
    op's operand) against the level-by-level kernels: the same logL, the
    same per-pattern values and the same gradient (the pre-order pass reads
    the stored partials), bit for bit, on a tree with ambiguous tips, two
    tiles and a ragged tail."""
    from paper_2606_27607_gb300 import TreeLikelihood
    w = codon_workload(37, 2 * 128 + 45)
    rng = np.random.default_rng(8)
    w.tips = w.tips.copy()
    w.tips[rng.random(w.tips.shape) < 0.03] = 61
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("TL_TC_FUSED", fused)
        tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 61, 4, prec)
        try:
            tl.set_tips(w.tips)
            tl.set_model("gy94", w.params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_pattern_weights(w.pattern_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            logl, site = tl.loglik(site=True)
            _, g = tl.gradient()
            launches = tl.inst.launch_count()
        finally:
            tl.close()
        out[fused] = (logl, site, g, launches)
    assert out["1"][0] == out["0"][0]
    assert np.array_equal(out["1"][1], out["0"][1])
    assert np.array_equal(out["1"][2], out["0"][2])
    assert out["1"][3] < out["0"][3]      # one post-order launch instead of one per level
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    assert abs(out["1"][0] - want_l) <= 1e-5 * abs(want_l)


@pytest.mark.slow
def test_codon_128x20k_split_partials_full_size():
    """The benchmark's codon configuration (GY94, 128 taxa x 20,000 patterns)
    with split partials, every kernel launched over all patterns: per-pattern
    log-likelihoods on 300 sampled patterns (the ragged tail among them)
    within 2^-20 (N - 1) of the oracle, and, with pattern weights that select
    those patterns, logL and every branch derivative against the oracle on
    them alone (per-component bound)."""
    import dataclasses

    from oracle import gradient as og
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload("gy94_128x20k")
    rng = np.random.default_rng(12)
    idx = np.sort(rng.choice(w.n_patterns, 300, replace=False))
    idx[-1] = w.n_patterns - 1
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    logl, site = run(w, "tf32x3", site=True)
    _, want_site = op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                     w.tips, patterns=idx)
    assert np.max(np.abs(site[idx] - want_site)) <= 2.0 ** -20 * 127
    wt = np.zeros(w.n_patterns)
    wt[idx] = 1.0
    small = dataclasses.replace(w, tips=w.tips[:, idx], pattern_weights=np.ones(len(idx)))
    want_l, _ = op.loglik(small.tree, Q, pi, w.rates, w.cat_weights, small.pattern_weights,
                          small.tips)
    want_g = og.branch_gradient(small.tree, Q, pi, w.rates, w.cat_weights, small.pattern_weights,
                                small.tips)
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 61, 4, "tf32x3")
    try:
        tl.set_tips(w.tips)
        tl.set_model("gy94", w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(wt)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        lsel, g = tl.gradient()
    finally:
        tl.close()
    assert abs(lsel - want_l) <= 1e-5 * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-3)
