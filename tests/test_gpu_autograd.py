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


def per_component(got, want):
    scale = np.max(np.abs(want))
    return np.max(np.abs(got - want) / np.maximum(np.abs(want), 1e-3 * scale))


@pytest.mark.parametrize("prec,tol,shape", [("f64", 1e-10, (6, 120)), ("tf32x3", 1e-3, (6, 120)),
                                            ("tf32x3", 1e-3, (10, 200))])
def test_codon_subst_gradient_matches_oracle(prec, tol, shape):
    """dlogL/dkappa and dlogL/domega for GY94 (one pre-order pass per
    parameter with dP/dtheta) on the FP64 generic path and on the split
    tensor-core path, each component against the oracle."""
    w = synth.workload("gy94_64x5k", n_tips=shape[0], n_patterns=shape[1])
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    want = og.subst_gradient(w.tree, Q, dQ, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    tl = make(w, prec, 61)
    try:
        tl.loglik()
        got = tl.subst_gradient()
    finally:
        tl.close()
    assert per_component(got, want) <= tol, (got, want)


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
        assert abs(float(y.detach()) - want_l) <= 1e-11 * abs(want_l)
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


def sampled(w, n=300, seed=5):
    """The workload with weight 1 on n sampled patterns and 0 elsewhere: the
    full-size launch computes a logL and gradient the oracle can evaluate on
    those n patterns alone."""
    import dataclasses
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(w.n_patterns, n, replace=False))
    idx[-1] = w.n_patterns - 1           # the ragged tail
    wt = np.zeros(w.n_patterns)
    wt[idx] = 1.0
    small = dataclasses.replace(w, tips=w.tips[:, idx], pattern_weights=np.ones(n))
    return dataclasses.replace(w, pattern_weights=wt), small


@pytest.mark.slow
@pytest.mark.parametrize("name,prec", [("gtr_1024x50k", "f32"), ("gy94_64x5k", "tf32x3")])
def test_autograd_full_size_sampled_patterns(name, prec):
    """The autograd Function at the benchmark's full sizes (every kernel
    launched over all patterns and the whole tree), with pattern weights
    that select 300 patterns: logL, all branch-length and substitution
    gradients against the oracle on those patterns; central differences of
    the FP64 GPU path (h = 1e-6) for a few components."""
    import torch

    from paper_2606_27607_gb300 import LogLikelihood
    w, small = sampled(synth.workload(name))
    S = w.n_states
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(small.tree, Q, pi, small.rates, small.cat_weights,
                          small.pattern_weights, small.tips)
    want_gt = og.branch_gradient(small.tree, Q, pi, small.rates, small.cat_weights,
                                 small.pattern_weights, small.tips)
    want_gk = og.subst_gradient(small.tree, Q, dQ, pi, small.rates, small.cat_weights,
                                small.pattern_weights, small.tips)
    tl = make(w, prec, S)
    try:
        t = torch.tensor(w.tree.edge_len[:-1], dtype=torch.float64, requires_grad=True)
        th = torch.tensor(w.params, dtype=torch.float64, requires_grad=True)
        y = LogLikelihood.apply(t, th, tl, w.model, w.freqs)
        y.backward()
        gt, gk = t.grad.numpy(), th.grad.numpy()
    finally:
        tl.close()
    assert abs(float(y.detach()) - want_l) <= 1e-5 * abs(want_l)
    wt = want_gt[:-1]
    assert per_component(gt, wt) <= 1e-3
    assert per_component(gk, want_gk) <= 1e-3
    # central differences of the FP64 GPU path at full size
    t64 = make(w, "f64", S)
    try:
        h = 1e-6
        base_t, base_k = w.tree.edge_len[:-1].copy(), np.array(w.params, float)

        def f(tt, kk):
            return float(LogLikelihood.apply(torch.tensor(tt), torch.tensor(kk), t64, w.model,
                                             w.freqs).detach())

        for v in (0, int(np.argmax(np.abs(wt))), len(base_t) - 1):
            tp, tm = base_t.copy(), base_t.copy()
            tp[v] += h
            tm[v] -= h
            fd = (f(tp, base_k) - f(tm, base_k)) / (2 * h)
            assert abs(fd - gt[v]) <= 1e-3 * max(abs(fd), 1e-3 * np.max(np.abs(wt))), (v, fd, gt[v])
        kp, km = base_k.copy(), base_k.copy()
        kp[0] += h
        km[0] -= h
        fd = (f(base_t, kp) - f(base_t, km)) / (2 * h)
        assert abs(fd - gk[0]) <= 1e-3 * max(abs(fd), 1e-3 * np.max(np.abs(gk)))
    finally:
        t64.close()


def test_two_forwards_then_one_backward():
    """loss = f(t1) + f(t2) on one instance: each backward must see its own
    forward's partials, not those of the last evaluation on the instance."""
    import torch

    from paper_2606_27607_gb300 import LogLikelihood
    w = synth.workload("hky_8x1000", n_tips=10, n_patterns=200)
    Q, pi, dQ = om.build(w.model, w.params, w.freqs)
    t1 = w.tree.edge_len[:-1].copy()
    t2 = t1 * np.linspace(0.5, 1.7, len(t1))
    want = []
    for tt in (t1, t2):
        full = np.append(tt, 0.0)
        tree = synth.Tree(w.tree.n_tips, w.tree.children, w.tree.parent, full)
        want.append(og.branch_gradient(tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                       w.tips)[:-1])
    tl = make(w, "f64", 4)
    try:
        a = torch.tensor(t1, dtype=torch.float64, requires_grad=True)
        b = torch.tensor(t2, dtype=torch.float64, requires_grad=True)
        th = torch.tensor(w.params, dtype=torch.float64)
        loss = LogLikelihood.apply(a, th, tl, "hky", w.freqs) + \
            2.0 * LogLikelihood.apply(b, th, tl, "hky", w.freqs)
        loss.backward()
    finally:
        tl.close()
    assert np.allclose(a.grad.numpy(), want[0], rtol=1e-10, atol=1e-10)
    assert np.allclose(b.grad.numpy(), 2.0 * want[1], rtol=1e-10, atol=1e-10)
