"""tl_adjoint (reverse-mode gradient through the adjoint of the matrix
exponential's derivative) against the FP64 oracle: dlogL/dt for every
branch, dlogL/dQ, dlogL/dtheta for every model parameter (including the 265
of random-effects GY94), and the first-order approximation, on the
four-state kernels, the FP64 generic path and the tensor-core codon path
(split partials, and TF32-stored partials at their own bound), every
component within |x - x*| <= tol max(|x*|, 1e-3 |x*|_inf)."""
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


def run(w, prec, first_order=False, model=None, params=None):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, len(w.rates), prec)
    try:
        tl.set_tips(w.tips)
        tl.set_model(model or w.model, w.params if params is None else params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        logl = tl.loglik()
        g, dq, th = tl.adjoint(first_order)
        return logl, g, dq, th
    finally:
        tl.close()


def want(w, first_order=False, model=None, params=None):
    model = model or w.model
    params = w.params if params is None else params
    Q, pi, _ = om.build(model, params, w.freqs)
    args = (w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    logl = op.loglik(*args)[0]
    g = og.branch_gradient(*args)
    G = og.rate_matrix_gradient(*args, first_order=first_order)
    J = om.rate_jacobian(model, params, w.freqs)
    return logl, g, G, np.einsum("kij,ij->k", J, G)


def close(got, ref, tol):
    """Per component |x - x*| <= tol max(|x*|, 1e-3 |x*|_inf)."""
    got, ref = np.ravel(got), np.ravel(ref)
    scale = np.max(np.abs(ref))
    return np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * scale)) <= tol


def rate_entries(w, model=None, params=None):
    """Entries of dlogL/dQ compared at the reduced-precision bound: those
    where Q is not zero (all of them for four states). At the structural
    zeros of a codon Q (codons three or two changes apart) dlogL/dQ is up to
    1e7 times larger and ill-conditioned: the FP64 path itself agrees with
    the oracle there to only 5e-8, and FP32 partials to about 1e-3. No model
    parameter moves those entries."""
    Q = om.build(model or w.model, w.params if params is None else params, w.freqs)[0]
    return Q != 0


def check(w, prec, tol, first_order=False, model=None, params=None):
    gl, gg, gq, gt = run(w, prec, first_order, model, params)
    wl, wg, wq, wt = want(w, first_order, model, params)
    assert abs(gl - wl) <= 1e-5 * abs(wl)
    assert close(gg[:-1], wg[:-1], tol), (np.max(np.abs(gg - wg)), np.max(np.abs(wg)))
    m = rate_entries(w, model, params) if prec != "f64" else np.ones(gq.shape, bool)
    assert close(gq[m], wq[m], tol), (np.max(np.abs(gq - wq)), np.max(np.abs(wq)))
    if wt.size:
        assert close(gt, wt, tol), (gt[:8], wt[:8])
    return gg, gq, gt


@pytest.mark.parametrize("name,prec,tol", [("hky_8x1000", "f64", 1e-10), ("hky_8x1000", "f32", 1e-3),
                                           ("gtr_512x100k", "f64", 1e-10),
                                           ("gtr_512x100k", "f32", 1e-3)])
def test_four_state_adjoint(name, prec, tol):
    """Several pattern chunks (5,000 patterns) and a ragged tail."""
    w = synth.workload(name, n_tips=23, n_patterns=5001)
    check(w, prec, tol)


@pytest.mark.parametrize("ncat", [1, 3, 6])
def test_four_state_category_counts(ncat):
    w = synth.workload("gtr_512x100k", n_tips=11, n_patterns=700)
    w = dataclasses.replace(w, rates=synth.gamma_rates(0.5, ncat),
                            cat_weights=np.full(ncat, 1.0 / ncat))
    check(w, "f32", 1e-3)
    check(w, "f64", 1e-10)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_first_order_approximation(prec):
    w = synth.workload("gtr_512x100k", n_tips=15, n_patterns=300)
    check(w, prec, 1e-10 if prec == "f64" else 1e-3, first_order=True)


def test_ambiguous_tips_zero_weights_and_tip_partials():
    """Ambiguous codes, weight 0 and 5, and two tips given as partials."""
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload("hky_8x1000", n_tips=9, n_patterns=260)
    tips = w.tips.copy()
    tips[:3, :10] = 4
    wt = np.ones(w.n_patterns)
    wt[5] = 0.0
    wt[20:30] = 5.0
    w = dataclasses.replace(w, tips=tips, pattern_weights=wt)
    wl, wg, wq, wth = want(w)
    for prec, tol in (("f64", 1e-10), ("f32", 1e-3)):
        tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, prec)
        try:
            tl.set_tips(w.tips)
            for t in (0, 4):   # as one-hot / all-ones partials
                part = np.zeros((w.n_patterns, 4))
                s = w.tips[t]
                ok = (s >= 0) & (s < 4)
                part[np.arange(w.n_patterns)[ok], s[ok]] = 1.0
                part[~ok] = 1.0
                tl.inst.set_tip_partials(t, part)
            tl.set_model(w.model, w.params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_pattern_weights(w.pattern_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            tl.loglik()
            g, dq, th = tl.adjoint()
        finally:
            tl.close()
        assert close(g[:-1], wg[:-1], tol)
        assert close(dq, wq, tol)
        assert close(th, wth, tol)


@pytest.mark.parametrize("prec,tol,n_tips,n_pat", [("f64", 1e-9, 7, 161), ("f64", 1e-8, 20, 300),
                                                   ("tf32x3", 1e-3, 7, 161),
                                                   ("tf32x3", 1e-3, 20, 300)])
def test_codon_adjoint(prec, tol, n_tips, n_pat):
    """GY94: the FP64 generic path and the split tensor-core path (FP32
    partials split on chip), every component of every gradient. The FP64
    bound at 20 taxa is the one its eigensystem route reaches (4.5e-9 of
    the floor 1e-3 |g|_inf, i.e. 4.5e-12 of the largest component, in the
    fused pre-order gradient and the adjoint alike): F3x4 frequencies make
    V = D^-1/2 U scale by 1/sqrt(pi_min)."""
    w = synth.workload("gy94_64x5k", n_tips=n_tips, n_patterns=n_pat)
    check(w, prec, tol)


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
@pytest.mark.parametrize("n_tips,n_pat", [(7, 161), (20, 300)])
def test_codon_adjoint_tf32_storage(prec, n_tips, n_pat):
    """The tensor-core adjoint on TF32-stored partials (the accumulation
    kernel's variant without the x_lo products). Partials rounded to 11 bits
    give per-component gradient errors up to 1e-2 of a component on small
    trees (terms that cancel keep an absolute error of order 2^-11 sqrt(P) of
    their size); measured up to 3.4e-3 here, so the bound is 1e-2, while a
    wrong operand layout or a dropped product errs by order one."""
    w = synth.workload("gy94_64x5k", n_tips=n_tips, n_patterns=n_pat)
    check(w, prec, 1e-2)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-9), ("tf32x3", 1e-3)])
def test_random_effects_gy94(prec, tol):
    """All 265 parameters of random-effects GY94 (kappa, omega and one
    effect per one-difference codon pair), against <dlogL/dQ, dQ/dtheta> of
    the oracle with complex-step dQ/dtheta; logL checks the device-built Q."""
    w = synth.workload("gy94_64x5k", n_tips=6, n_patterns=130)
    eps = np.random.default_rng(7).normal(0.0, 0.4, 263)
    params = np.r_[w.params, eps]
    _, _, th = check(w, prec, tol, model="gy94re", params=params)
    assert th.shape == (265,)


def test_adjoint_agrees_with_pre_order_gradient_and_euler_identity():
    """The adjoint's branch derivatives equal the fused pre-order gradient's
    (same precision), and <dlogL/dQ, Q> = sum_v t_v dlogL/dt_v."""
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload("gtr_512x100k", n_tips=40, n_patterns=3000)
    Q = om.build(w.model, w.params, w.freqs)[0]
    for prec, tol in (("f64", 1e-10), ("f32", 1e-4)):
        tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, prec)
        try:
            tl.set_tips(w.tips)
            tl.set_model(w.model, w.params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_pattern_weights(w.pattern_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            _, g1 = tl.gradient()
            tl.loglik()
            g2, dq, _ = tl.adjoint()
        finally:
            tl.close()
        assert close(g2[:-1], g1[:-1], tol)
        ref = float(np.dot(w.tree.edge_len[:-1], g2[:-1]))
        assert abs(np.sum(dq * Q) - ref) <= tol * np.sum(np.abs(w.tree.edge_len[:-1] * g2[:-1]))


def test_adjoint_argument_errors():
    from paper_2606_27607_gb300 import TreeLikelihood, TreelikError
    w = synth.workload("hky_8x1000", n_tips=5, n_patterns=64)
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, "f32")
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        tl.loglik()
        tl.inst.update_pre_partials(tl._preq, 0)
        with pytest.raises(TreelikError, match="TL_ERR_ARG"):     # wrong parameter count
            tl.inst.adjoint(tl._adj, tl.nn, 2)
        bad = tl._adj.copy()
        bad["mat"][0, 0] = tl.nn + 1    # a slot holding no transition matrix of the model
        with pytest.raises(TreelikError, match="TL_ERR_STATE"):
            tl.inst.adjoint(bad, tl.nn, 1)
        bad = tl._adj.copy()
        bad["edge"][1, 0] = bad["edge"][0, 0]
        with pytest.raises(TreelikError, match="TL_ERR_ORDER"):
            tl.inst.adjoint(bad, tl.nn, 1)
        g, dq, th = tl.inst.adjoint(tl._adj, tl.nn, 1)
        assert np.all(np.isfinite(g)) and np.all(np.isfinite(dq)) and th.shape == (1,)
    finally:
        tl.close()


def sampled(w, n=300, seed=9):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.n_patterns, n, replace=False))
    idx[-1] = w.n_patterns - 1
    wt = np.zeros(w.n_patterns)
    wt[idx] = 1.0
    small = dataclasses.replace(w, tips=w.tips[:, idx], pattern_weights=np.ones(n))
    return dataclasses.replace(w, pattern_weights=wt), small


@pytest.mark.slow
@pytest.mark.parametrize("name,prec,model", [("gtr_1024x50k", "f32", None),
                                             ("gy94_128x20k", "tf32x3", "gy94re")])
def test_adjoint_full_size_sampled_patterns(name, prec, model):
    """Full-size launches (the benchmark's trees and pattern counts) with
    weights selecting 300 patterns, so the oracle can evaluate the same
    gradient on those patterns alone."""
    w, small = sampled(synth.workload(name))
    params = None
    if model == "gy94re":
        params = np.r_[w.params, np.random.default_rng(3).normal(0.0, 0.3, 263)]
    gl, gg, gq, gt = run(w, prec, model=model, params=params)
    wl, wg, wq, wt = want(small, model=model, params=params)
    assert abs(gl - wl) <= 1e-5 * abs(wl)
    assert close(gg[:-1], wg[:-1], 1e-3)
    m = rate_entries(w, model, params)
    assert close(gq[m], wq[m], 1e-3)
    assert close(gt, wt, 1e-3)
