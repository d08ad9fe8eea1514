"""Substitution-parameter gradients (kappa, omega, GTR exchangeabilities) and
the autograd Function, against the FP64 oracle (exact Frechet derivative of
the matrix exponential) and central finite differences of the GPU FP64 path."""
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


def make(w, prec, S):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, S, 4, prec)
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_pattern_weights(w.pattern_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    return tl


@pytest.mark.parametrize("model,prec,tol", [("hky", "f64", 1e-11), ("hky", "f32", 1e-3),
                                            ("gtr", "f64", 1e-11), ("gtr", "f32", 1e-3)])
def test_subst_gradient_matches_oracle(model, prec, tol):
    if model == "hky":
        w = synth.workload("hky_8x1000", n_tips=20, n_patterns=500)
    else:
        w = synth.workload("gtr_512x100k", n_tips=25, n_patterns=400)
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    want = og.subst_gradient(w.tree, Q, dQ, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = make(w, prec, 4)
    try:
        tl.loglik()
        got = tl.subst_gradient()
    finally:
        tl.close()
    scale = np.max(np.abs(want))
    err = np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * scale)
    assert np.max(err) <= tol, (got, want)


def test_codon_subst_gradient_tf32():
    w = synth.workload("gy94_64x5k", n_tips=10, n_patterns=200)
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    want = og.subst_gradient(w.tree, Q, dQ, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = make(w, "tf32", 61)
    try:
        tl.loglik()
        got = tl.subst_gradient()
    finally:
        tl.close()
    assert np.linalg.norm(got - want) <= 1e-3 * np.linalg.norm(want), (got, want)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("tf32x2", 1e-3)])
def test_codon_subst_gradient_matches_oracle(prec, tol):
    """dlogL/dkappa and dlogL/domega for GY94 on the FP64 generic path and on
    the split-TF32 tensor-core path."""
    w = synth.workload("gy94_64x5k", n_tips=6, n_patterns=120)
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    want = og.subst_gradient(w.tree, Q, dQ, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = make(w, prec, 61)
    try:
        tl.loglik()
        got = tl.subst_gradient()
    finally:
        tl.close()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want)), (got, want)


def test_autograd_function_matches_oracle_and_finite_differences():
    import torch

    from paper_2606_27607_gb300 import LogLikelihood
    w = synth.workload("hky_8x1000", n_tips=12, n_patterns=300)
    tl = make(w, "f64", 4)
    try:
        t = torch.tensor(w.tree.edge_len[:-1], dtype=torch.float64, requires_grad=True)
        th = torch.tensor(w.params, dtype=torch.float64, requires_grad=True)
        y = LogLikelihood.apply(t, th, tl, "hky", w.freqs)
        y.backward()
        Q, pi, dQ = om.build(w.model, w.params, w.freqs)
        want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
        want_gt = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                     w.tips)
        want_gk = og.subst_gradient(w.tree, Q, dQ, pi, w.rates, w.cat_weights,
                                    w.pattern_weights, w.tips)
        assert abs(float(y) - want_l) <= 1e-11 * abs(want_l)
        assert np.allclose(t.grad.numpy(), want_gt[:-1], rtol=1e-10, atol=1e-10)
        assert np.allclose(th.grad.numpy(), want_gk, rtol=1e-10, atol=1e-10)
        # central differences of the GPU FP64 path itself, h = 1e-6
        h = 1e-6
        f = lambda tt, kk: float(LogLikelihood.apply(torch.tensor(tt), torch.tensor(kk), tl, "hky",
                                                     w.freqs))
        t0, k0 = w.tree.edge_len[:-1].copy(), np.array(w.params, float)
        for v in (0, 5, 13, 20):
            tp, tm = t0.copy(), t0.copy()
            tp[v] += h
            tm[v] -= h
            fd = (f(tp, k0) - f(tm, k0)) / (2 * h)
            assert abs(fd - t.grad.numpy()[v]) <= 1e-5 * max(1.0, abs(fd))
        fd = (f(t0, k0 + h) - f(t0, k0 - h)) / (2 * h)
        assert abs(fd - th.grad.numpy()[0]) <= 1e-5 * max(1.0, abs(fd))
    finally:
        tl.close()
