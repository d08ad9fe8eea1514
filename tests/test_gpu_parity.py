"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the benchmark spec for this path): FP64 path relative error
<= 1e-11 on logL and gradients; reduced precision <= 1e-5 on logL and
<= 1e-3 on gradients. A gradient component is compared as
|g - g*| <= tol * max(|g*|, 1e-3 * max|g*|) since a pure relative error is
ill-posed for components near zero. Tip compression (states vs one-hot tip
partials) and operation order must be bit-exact.
"""
import numpy as np
import pytest

import synth
from oracle import gradient as og, model as om, pruning as op

pytestmark = pytest.mark.gpu

TOL = {"f64": (1e-11, 1e-11), "f32": (1e-5, 1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import build
    build.build()


def oracle_run(w, grad=True):
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    logl, site = op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                           w.tips) if grad else None
    return logl, site, g


def gpu_run(w, prec, grad=True, site=False, tl_kwargs=None):
    from paper_2606_27607_gb300 import TreeLikelihood
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, w.n_states, len(w.rates), prec,
                        **(tl_kwargs or {}))
    try:
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_pattern_weights(w.pattern_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        if grad:
            logl, g = tl.gradient()
            s = None
        else:
            g = None
            if site:
                logl, s = tl.loglik(site=True)
            else:
                logl, s = tl.loglik(), None
        return logl, s, g
    finally:
        tl.close()


def assert_grad_close(g, want, tol):
    scale = np.max(np.abs(want))
    den = np.maximum(np.abs(want), 1e-3 * scale)
    err = np.abs(g - want) / den
    assert np.max(err) <= tol, (np.max(err), int(np.argmax(err)))


def small_gtr(n_tips=40, n_patterns=1000 + 17, config=1, amb=0.02):
    w = synth.workload("gtr_512x100k", n_tips=n_tips, n_patterns=n_patterns)
    rng = np.random.default_rng(config + 100)
    mask = rng.random(w.tips.shape) < amb
    w.tips = w.tips.copy()
    w.tips[mask] = 4  # ambiguous code
    w.pattern_weights = rng.integers(1, 4, size=w.n_patterns).astype(float)
    return w


# ---------------------------------------------------------------------------
# model, eigensystem and transition matrices (a1, a2, a6)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["hky", "gtr", "gy94"])
def test_device_model_matches_oracle(kind):
    from paper_2606_27607_gb300 import Instance
    rng = np.random.default_rng(5)
    if kind == "hky":
        params, freqs = [2.5], rng.dirichlet(np.ones(4))
        S = 4
    elif kind == "gtr":
        params, freqs = rng.dirichlet(np.ones(6)) * 6, rng.dirichlet(np.ones(4))
        S = 4
    else:
        params, freqs = [2.0, 0.3], np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
        S = 61
    Q, pi, dQ = om.build(kind, params, freqs)
    with Instance(4, 8, S, 4, 4, 10, 1, "f64") as inst:
        inst.set_model(0, kind, params, freqs)
        Qg, pig, dQg = inst.get_model(0)
        assert np.allclose(Qg, Q, rtol=0, atol=1e-14 * np.abs(Q).max())
        assert np.allclose(pig, pi, rtol=1e-14, atol=0)
        assert len(dQg) == len(dQ)
        for a, b in zip(dQg, dQ):
            assert np.allclose(a, b, rtol=0, atol=1e-13 * max(1.0, np.abs(b).max()))
        rates = synth.gamma_rates(0.5)
        inst.set_category_rates(rates)
        t = np.array([0.0, 0.01, 0.1, 0.7, 3.0])
        inst.update_matrices(0, np.arange(5), t, np.arange(5) + 5)
        for b, tb in enumerate(t):
            P = inst.get_matrix(b)
            dP = inst.get_matrix(5 + b)
            for r, rho in enumerate(rates):
                want = op.transition_matrices(Q, np.array([tb]), [rho])[0, 0]
                assert np.allclose(P[r], want, rtol=0, atol=1e-13), (b, r)
                assert np.allclose(dP[r], rho * Q @ want, rtol=0, atol=1e-12 * max(1, rho))


@pytest.mark.parametrize("prec", ["tf32", "tf32x2"])
def test_codon_matrices_of_tf32_instances(prec):
    """A TF32 instance forms P and dP/dt with a double-float S^3 product:
    each entry within 2^-44 of the sum of its terms' magnitudes,
    S * max|V| * max|Vinv| * max|e| (a factor 16 above the 2^-48 the
    arithmetic keeps per term)."""
    from paper_2606_27607_gb300 import Instance
    rng = np.random.default_rng(11)
    params, freqs = [2.0, 0.3], np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
    Q, pi, _ = om.build("gy94", params, freqs)
    S = 61
    rates = synth.gamma_rates(0.5)
    t = np.array([0.0, 0.01, 0.1, 0.7, 3.0])
    d = np.sqrt(pi)
    A = d[:, None] * Q / d[None, :]
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    vmax, vimax = 1.0 / d.min(), d.max()
    with Instance(4, 8, S, 4, 4, 10, 1, prec) as inst:
        inst.set_model(0, "gy94", params, freqs)
        inst.set_category_rates(rates)
        inst.update_matrices(0, np.arange(5), t, np.arange(5) + 5)
        for b, tb in enumerate(t):
            P, dP = inst.get_matrix(b), inst.get_matrix(5 + b)
            for r, rho in enumerate(rates):
                want = op.transition_matrices(Q, np.array([tb]), [rho])[0, 0]
                emax = np.abs(np.expm1(lam * rho * tb)).max()
                demax = np.abs(rho * lam * np.exp(lam * rho * tb)).max()
                tol_p = S * vmax * vimax * emax * 2.0 ** -44 + 1e-13
                tol_d = S * vmax * vimax * demax * 2.0 ** -44 + 1e-12 * max(1, rho)
                assert np.abs(P[r] - want).max() <= tol_p, (b, r)
                assert np.abs(dP[r] - rho * Q @ want).max() <= tol_d, (b, r)


@pytest.mark.parametrize("case", ["gy94_degenerate", "rev40"])
def test_eigensystem_above_32_states(case):
    """Above 32 states the FP64 eigensystem comes from FP32 Jacobi, the
    simultaneous-rotation refinement and, where eigenvalues are too close
    for it, FP64 Jacobi sweeps. Uniform codon frequencies with kappa = omega
    = 1 give a spectrum of highly repeated eigenvalues (every pair of the
    repeated ones left to the sweeps); a 40-state general reversible model a
    generic one. P against the oracle at the FP64 path's tolerance."""
    from paper_2606_27607_gb300 import Instance
    rng = np.random.default_rng(17)
    if case == "gy94_degenerate":
        kind, S = "gy94", 61
        params, freqs = [1.0, 1.0], np.full((3, 4), 0.25)
    else:
        kind, S = "rev", 40
        ex = rng.exponential(1.0, size=(S, S))
        params, freqs = 0.5 * (ex + ex.T), rng.dirichlet(np.ones(S))
    Q, pi, _ = om.build(kind, params, freqs)
    d = np.sqrt(pi)
    lam = np.linalg.eigvalsh(0.5 * (d[:, None] * Q / d[None, :] + (d[:, None] * Q / d[None, :]).T))
    if case == "gy94_degenerate":
        assert np.sum(np.diff(np.sort(lam)) < 1e-9 * np.abs(lam).max()) > 10
    with Instance(4, 8, S, 4, 4, 10, 1, "f64") as inst:
        inst.set_model(0, kind, params, freqs)
        rates = synth.gamma_rates(0.5)
        inst.set_category_rates(rates)
        t = np.array([0.0, 0.01, 0.1, 0.7, 3.0])
        inst.update_matrices(0, np.arange(5), t, np.arange(5) + 5)
        for b, tb in enumerate(t):
            P, dP = inst.get_matrix(b), inst.get_matrix(5 + b)
            for r, rho in enumerate(rates):
                want = op.transition_matrices(Q, np.array([tb]), [rho])[0, 0]
                assert np.abs(P[r] - want).max() <= 1e-13, (b, r)
                assert np.abs(dP[r] - rho * Q @ want).max() <= 1e-12 * max(1, rho), (b, r)


def test_set_eigen_and_rate_matrix_paths():
    from paper_2606_27607_gb300 import Instance
    pi = np.array([0.1, 0.2, 0.3, 0.4])
    Q, _ = om.gtr([1, 2, 3, 4, 5, 6], pi)
    lam, V = np.linalg.eig(Q)
    Vi = np.linalg.inv(V)
    with Instance(4, 8, 4, 1, 4, 4, 2, "f64") as inst:
        inst.set_eigen(0, V.real, Vi.real, lam.real, pi)
        inst.set_rate_matrix(1, Q, pi)
        inst.set_category_rates([1.0])
        inst.update_matrices(0, [0], [0.3])
        inst.update_matrices(1, [1], [0.3])
        want = op.transition_matrices(Q, np.array([0.3]), [1.0])[0, 0]
        assert np.allclose(inst.get_matrix(0)[0], want, atol=1e-13)
        assert np.allclose(inst.get_matrix(1)[0], want, atol=1e-13)


# ---------------------------------------------------------------------------
# likelihood and gradient (a3-a5, a7-a8)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hky_8x1000_matches_oracle(prec):
    w = synth.workload("hky_8x1000")
    want_l, _, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, prec)
    tl, tg = TOL[prec]
    assert abs(logl - want_l) <= tl * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], tg)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("n_tips,n_pat", [(2, 33), (3, 1), (40, 1017), (150, 2500)])
def test_gtr_sizes_match_oracle(prec, n_tips, n_pat):
    w = small_gtr(n_tips, n_pat)
    want_l, want_site, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, prec)
    tl, tg = TOL[prec]
    assert abs(logl - want_l) <= tl * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], tg)
    _, site, _ = gpu_run(w, prec, grad=False, site=True)
    assert np.allclose(site, want_site, rtol=tl, atol=0)


def test_f64_without_rescaling_matches_oracle():
    w = small_gtr(30, 500)
    want_l, _, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, "f64", tl_kwargs={"scale": False})
    assert abs(logl - want_l) <= 1e-11 * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-11)


def test_deep_caterpillar_needs_rescaling_f32():
    # 700 tips in a caterpillar: FP32 partials underflow without rescaling
    n = 700
    children = np.zeros((n - 1, 2), dtype=np.int64)
    children[0] = (0, 1)
    for k in range(1, n - 1):
        children[k] = (n + k - 1, k + 1)
    w = synth.workload("hky_8x1000", n_patterns=64)
    rng = np.random.default_rng(4)
    w.tree = synth.Tree(n, children, -np.ones(2 * n - 1, dtype=np.int64),
                        np.r_[rng.exponential(0.1, 2 * n - 2), 0.0])
    w.tips = rng.integers(0, 4, size=(n, 64)).astype(np.int8)
    want_l, _, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, "f32")
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-3)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tip_states_equal_tip_partials_bit_exact(prec):
    from paper_2606_27607_gb300 import TreeLikelihood
    w = small_gtr(25, 300, amb=0.05)
    res = []
    for use_partials in (False, True):
        tl = TreeLikelihood(25, w.n_patterns, 4, 4, prec)
        if use_partials:
            for t in range(25):
                tl.inst.set_tip_partials(t, op.tip_partials(w.tips[t:t + 1], 4)[0])
        else:
            tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        res.append(tl.gradient())
        tl.close()
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])


def test_op_order_is_bit_exact():
    from paper_2606_27607_gb300 import TreeLikelihood, tree
    w = small_gtr(60, 700)
    tl = TreeLikelihood(60, w.n_patterns, 4, 4, "f32")
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    l1, g1 = tl.gradient()
    # a different valid order: post-order ops sorted by node depth (levels)
    post = tree.post_ops(w.tree.children, 60)
    depth = np.zeros(119, dtype=int)
    for k, (a, b) in enumerate(w.tree.children):
        depth[60 + k] = 1 + max(depth[a], depth[b])
    order = np.argsort(depth[post["dest"]], kind="stable")
    tl.inst.update_partials(post[order])
    l2 = tl.inst.root_loglik(118, 0)
    # and each op in its own call
    for o in post:
        tl.inst.update_partials(o[None])
    l3 = tl.inst.root_loglik(118, 0)
    assert l1 == l2 == l3
    g2 = tl.inst.pre_order_gradient(tl._pre, 119, 0)
    assert np.array_equal(g1, g2)
    tl.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_materialised_pre_partials_and_edge_derivatives(prec):
    from paper_2606_27607_gb300 import TreeLikelihood, tree
    w = small_gtr(30, 400)
    want_l, _, want_g = oracle_run(w)
    tl = TreeLikelihood(30, w.n_patterns, 4, 4, prec, store_pre=True)
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_pattern_weights(w.pattern_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    tl.update_matrices(True)
    tl.inst.update_partials(tl._post)
    pre = tree.pre_ops(w.tree.children, 30, tl.pre_base, with_edges=False, tip_pre=True)
    tl.inst.update_pre_partials(pre, 0)
    g = tl.inst.edge_derivatives(tree.edges(30, tl.pre_base), 59, 0)
    # pre- and post-order partials themselves, against the oracle's (each is
    # defined up to its per-pattern power-of-two scale: compare normalised)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    P = op.transition_matrices(Q, w.tree.edge_len, w.rates)
    tips = op.tip_partials(w.tips, 4)
    post, exps = op.post_order(w.tree.children, 30, P, tips, True)
    q, _ = og.pre_order(w.tree.children, 30, P, post, tips, pi, 4, True)
    rtol = 1e-13 if prec == "f64" else 2e-6
    for v in range(30, 59):
        got, e = tl.inst.get_partials(v)
        assert np.array_equal(e, sum(exps[k] for k in range(30, v + 1) if is_desc(w.tree, k, v)))
        assert np.allclose(got, post[v], rtol=rtol, atol=rtol * np.max(post[v]))
    for v in range(58):
        got, _ = tl.inst.get_partials(tl.pre_base + v)
        a = got / got.max(axis=(0, 2), keepdims=True)
        b = q[v] / q[v].max(axis=(0, 2), keepdims=True)
        assert np.allclose(a, b, rtol=rtol, atol=rtol), v
    tl.close()
    assert_grad_close(g[:-1], want_g[:-1], TOL[prec][1])


def is_desc(tree, k, v):
    """internal node k is v or lies below v"""
    while k != v and k < 2 * tree.n_tips - 2:
        k = int(np.nonzero(tree.children == k)[0][0]) + tree.n_tips
    return k == v


def test_codon_f64_generic_matches_oracle():
    w = synth.workload("gy94_64x5k", n_tips=6, n_patterns=45)
    want_l, _, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, "f64")
    assert abs(logl - want_l) <= 1e-11 * abs(want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-11)


# ---------------------------------------------------------------------------
# full-size configurations (sampled or property checks)
# ---------------------------------------------------------------------------

@pytest.mark.slow
def test_gtr_512x100k_f32_full_size():
    w = synth.workload("gtr_512x100k")
    logl, site, _ = gpu_run(w, "f32", grad=False, site=True)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(w.n_patterns, 600, replace=False))
    idx[-1] = w.n_patterns - 1   # the ragged tail
    _, want_site = op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights,
                                     w.pattern_weights, w.tips, patterns=idx)
    assert np.allclose(site[idx], want_site, rtol=1e-5, atol=0)
    assert abs(logl - np.sum(site)) <= 1e-9 * abs(logl)
    want_l, _ = op.loglik_chunked(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    assert abs(logl - want_l) <= 1e-5 * abs(want_l)


@pytest.mark.slow
def test_gtr_512x100k_f32_gradient_full_size_sampled():
    """The benchmark's headline configuration (512 taxa x 100,000 patterns,
    FP32 partials) with every kernel launched over all patterns: pattern
    weights select 300 patterns (the ragged tail among them) and are 0
    elsewhere, so the oracle evaluates logL and all 1,022 branch derivatives
    on those patterns alone; every component meets the reduced-precision
    bound. With weight 1 everywhere, the FP32 gradient matches the FP64 GPU
    path (itself oracle-checked) in the same per-component bound."""
    import dataclasses
    w = synth.workload("gtr_512x100k")
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(w.n_patterns, 300, replace=False))
    idx[-1] = w.n_patterns - 1
    wt = np.zeros(w.n_patterns)
    wt[idx] = 1.0
    sel = dataclasses.replace(w, pattern_weights=wt)
    small = dataclasses.replace(w, tips=w.tips[:, idx], pattern_weights=np.ones(len(idx)))
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    want_l, _ = op.loglik(small.tree, Q, pi, w.rates, w.cat_weights, small.pattern_weights,
                          small.tips)
    want_g = og.branch_gradient(small.tree, Q, pi, w.rates, w.cat_weights,
                                small.pattern_weights, small.tips)
    logl, _, g = gpu_run(sel, "f32")
    assert abs(logl - want_l) <= 1e-5 * abs(want_l), (logl, want_l)
    assert_grad_close(g[:-1], want_g[:-1], 1e-3)
    l32, _, g32 = gpu_run(w, "f32")
    l64, _, g64 = gpu_run(w, "f64")
    assert abs(l32 - l64) <= 1e-5 * abs(l64)
    assert_grad_close(g32[:-1], g64[:-1], 1e-3)


# ---------------------------------------------------------------------------
# errors
# ---------------------------------------------------------------------------

def test_errors_are_reported():
    from paper_2606_27607_gb300 import Instance, TreelikError, tree
    w = small_gtr(8, 64)
    with Instance(8, 64, 4, 4, 14, 30, 1, "f32") as inst:
        for t in range(8):
            inst.set_tip_states(t, w.tips[t])
        with pytest.raises(TreelikError, match="TL_ERR_STATE"):
            inst.update_matrices(0, [0], [0.1])
        inst.set_model(0, "gtr", w.params, w.freqs)
        with pytest.raises(TreelikError, match="TL_ERR_NUMERIC"):
            inst.update_matrices(0, [0], [-1.0])
        inst.update_matrices(0, np.arange(15), w.tree.edge_len[:15])
        post = tree.post_ops(w.tree.children, 8)
        with pytest.raises(TreelikError, match="TL_ERR_ORDER"):
            inst.update_partials(post[::-1])
        bad = post.copy()
        bad[0]["child1"] = 99
        with pytest.raises(TreelikError, match="TL_ERR_INDEX"):
            inst.update_partials(bad)
        inst.update_partials(post)
        assert np.isfinite(inst.root_loglik(14))
    with pytest.raises(TreelikError, match="TL_ERR_UNSUPPORTED"):
        Instance(4, 10, 5, 4, 4, 4, 1, "f32")
    # a pattern with zero likelihood
    with Instance(2, 4, 4, 1, 1, 2, 1, "f64") as inst:
        inst.set_tip_partials(0, np.array([[1, 0, 0, 0]] * 3 + [[0, 0, 0, 0]], float))
        inst.set_tip_states(1, [0, 1, 2, 3])
        inst.set_model(0, "hky", [2.0], [0.25] * 4)
        inst.update_matrices(0, [0, 1], [0.1, 0.1])
        inst.update_partials(np.array([(2, 0, 0, 1, 1)], dtype=tree.OP_DTYPE))
        with pytest.raises(TreelikError, match="TL_ERR_NUMERIC"):
            inst.root_loglik(2)


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("ncat", [1, 3, 6, 8])
def test_category_counts_match_oracle(prec, ncat):
    """Other category counts than four take the runtime-R kernels (one lane
    per category for R < 4, eight lanes for R > 4) and the root/edge layouts
    with LPP = 1, 4 or 8: logL and every branch derivative against the
    oracle with the counts' own Gamma rates and unequal weights."""
    import synth
    w = synth.workload("gtr_512x100k", n_tips=23, n_patterns=517)
    rates = synth.gamma_rates(0.7, ncat)
    catw = np.linspace(1.0, 2.0, ncat)
    catw = catw / catw.sum()
    rates = rates / np.sum(rates * catw)
    w.rates, w.cat_weights = rates, catw
    want_l, _, want_g = oracle_run(w)
    logl, _, g = gpu_run(w, prec)
    tol_l, tol_g = (1e-11, 1e-10) if prec == "f64" else (1e-5, 1e-3)
    assert abs(logl - want_l) <= tol_l * abs(want_l), (logl, want_l)
    assert_grad_close(g, want_g, tol_g)


def test_async_double_buffered_tip_upload():
    """tl_set_tip_states_all_async: uploads into the second pool overlap the
    work queued before them, and each evaluation sees exactly the tips of
    its own upload (two alternating data sets, both pools reused several
    times) - bit-identical to the synchronous upload."""
    import torch
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload("gtr_512x100k", n_tips=30, n_patterns=1000 + 17)
    rng = np.random.default_rng(4)
    other = rng.integers(0, 4, size=w.tips.shape).astype(np.int8)
    sets = [torch.from_numpy(np.ascontiguousarray(t)).pin_memory() for t in (w.tips, other)]
    want = []
    for t in sets:
        tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, "f32")
        try:
            tl.inst.set_tip_states_all(t.numpy())
            tl.set_model(w.model, w.params, w.freqs)
            tl.set_rates(w.rates, w.cat_weights)
            tl.set_tree(w.tree.children, w.tree.edge_len)
            want.append(tl.gradient())
        finally:
            tl.close()
    tl = TreeLikelihood(w.tree.n_tips, w.n_patterns, 4, 4, "f32")
    try:
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        for k in range(6):
            tl.inst.set_tip_states_all_async(sets[k % 2].numpy())
            logl, g = tl.gradient()
            assert logl == want[k % 2][0]
            assert np.array_equal(g, want[k % 2][1])
    finally:
        tl.close()
