"""Pins of the FP64 oracle to things other than itself: closed forms,
brute force, invariants of reversible models and finite differences.

Each pin is chosen so that a plausible mistake (a transposed operand, a
dropped normaliser, kappa on the wrong pairs, a wrong sign in the pre-order
step, a missing rate in dP/dt) fails at least one test.
"""
import os
from types import SimpleNamespace

import numpy as np
import pytest
from scipy.linalg import expm

import synth
from oracle import brute, gradient, model, pruning

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# helpers (test-side tree surgery; no likelihood arithmetic)
# ----------------------------------------------------------------------------

def small_tree(n_tips, seed, mean=0.3):
    rng = np.random.default_rng(seed)
    return synth.yule_tree(n_tips, rng, mean)


def reroot(tree, edge_child, frac):
    """Same unrooted tree, root moved onto the edge above ``edge_child``
    (split frac : 1-frac). Tips keep their labels; internal nodes are
    relabelled in post-order."""
    n = tree.n_tips
    root = 2 * n - 2
    adj = {}

    def link(x, y, t):
        adj.setdefault(x, {})[y] = t
        adj.setdefault(y, {})[x] = t

    ra, rb = tree.children[root - n]
    for k, (a, b) in enumerate(tree.children):
        v = n + k
        if v == root:
            continue
        link(v, a, tree.edge_len[a])
        link(v, b, tree.edge_len[b])
    link(ra, rb, tree.edge_len[ra] + tree.edge_len[rb])
    x = edge_child
    if x in (ra, rb):
        y = rb if x == ra else ra
    else:
        y = int(tree.parent[x])
    L = adj[x][y]
    del adj[x][y], adj[y][x]
    NEW = -1
    link(NEW, x, frac * L)
    link(NEW, y, (1 - frac) * L)
    order, kids = [], {}
    stack = [(NEW, None, False)]
    while stack:
        v, par, done = stack.pop()
        if done:
            order.append(v)
            continue
        nb = [w for w in adj[v] if w != par]
        if not nb:
            continue
        assert len(nb) == 2
        kids[v] = nb
        stack.append((v, par, True))
        for w in reversed(nb):
            stack.append((w, v, False))
    label = {v: v for v in range(n)}
    for k, v in enumerate(order):
        label[v] = n + k
    children = np.zeros((n - 1, 2), dtype=np.int64)
    el = np.zeros(2 * n - 1)
    for v, (a, b) in kids.items():
        children[label[v] - n] = (label[a], label[b])
        el[label[a]] = adj[v][a]
        el[label[b]] = adj[v][b]
    return SimpleNamespace(n_tips=n, children=children, edge_len=el)


def rand_states(rng, n_tips, n_pat, S, amb_frac=0.05):
    s = rng.integers(0, S, size=(n_tips, n_pat))
    amb = rng.random((n_tips, n_pat)) < amb_frac
    s[amb] = S  # ambiguous code
    return s.astype(np.int8)


# ----------------------------------------------------------------------------
# Gamma rates (inputs) and substitution models
# ----------------------------------------------------------------------------

def test_gamma_rates_match_yang1994():
    ref = np.loadtxt(os.path.join(GOLDEN, "gamma_mean_alpha05.txt"))
    got = synth.gamma_rates(0.5, 4)
    assert np.allclose(got, ref, atol=6e-5)
    assert abs(got.sum() - 4.0) < 1e-12


def test_genetic_code_table():
    codons, amino = model.genetic_code()
    assert len(codons) == 61
    from collections import Counter
    sizes = sorted(Counter(amino).values())
    # standard code: L,S,R x6; A,G,P,T,V x4; I x3; F,Y,H,Q,N,K,D,E,C x2; M,W x1
    assert sizes == sorted([6] * 3 + [4] * 5 + [3] + [2] * 9 + [1] * 2)
    spell = {"".join(model.BASES[i] for i in c): a for c, a in zip(codons, amino)}
    for cod, aa in {"ATG": "M", "TGG": "W", "TTT": "F", "TTA": "L", "CTG": "L",
                    "AGA": "R", "CGT": "R", "AGC": "S", "TCA": "S", "ATA": "I",
                    "GAT": "D", "GAA": "E", "AAA": "K", "CAT": "H", "CAG": "Q",
                    "TGT": "C", "TAT": "Y", "AAC": "N", "GGG": "G", "GCC": "A",
                    "CCC": "P", "ACG": "T", "GTA": "V"}.items():
        assert spell[cod] == aa, cod
    for stop in ("TAA", "TAG", "TGA"):
        assert stop not in spell


def test_jc_and_k80_closed_forms():
    pi = np.full(4, 0.25)
    for t in (0.0, 0.05, 0.3, 2.0):
        Q, _ = model.hky(1.0, pi)
        P = expm(t * Q)
        e = np.exp(-4 * t / 3)
        assert np.allclose(np.diag(P), 0.25 + 0.75 * e, atol=1e-14)
        assert np.allclose(P[0, 1], 0.25 - 0.25 * e, atol=1e-14)
        k = 3.0
        Q, _ = model.hky(k, pi)
        P = expm(t * Q)
        e1 = np.exp(-4 * t / (k + 2))
        e2 = np.exp(-2 * t * (k + 1) / (k + 2))
        assert np.isclose(P[0, 0], 0.25 + 0.25 * e1 + 0.5 * e2, atol=1e-14)
        assert np.isclose(P[0, 2], 0.25 + 0.25 * e1 - 0.5 * e2, atol=1e-14)  # A->G
        assert np.isclose(P[1, 3], 0.25 + 0.25 * e1 - 0.5 * e2, atol=1e-14)  # C->T
        assert np.isclose(P[0, 1], 0.25 - 0.25 * e1, atol=1e-14)             # A->C
        assert np.isclose(P[2, 3], 0.25 - 0.25 * e1, atol=1e-14)             # G->T


def test_f81_closed_form_through_gtr():
    pi = np.array([0.1, 0.2, 0.3, 0.4])
    Q, _ = model.gtr(np.ones(6), pi)
    beta = 1.0 / (1.0 - np.sum(pi ** 2))
    for t in (0.01, 0.4, 3.0):
        P = expm(t * Q)
        e = np.exp(-beta * t)
        want = np.outer(np.ones(4), pi) * (1 - e) + np.eye(4) * e
        assert np.allclose(P, want, atol=1e-14)


def test_hky_is_gtr_special_case():
    pi = np.array([0.3, 0.2, 0.2, 0.3])
    Qh, dh = model.hky(2.5, pi)
    Qg, dg = model.gtr([1, 2.5, 1, 1, 2.5, 1], pi)
    assert np.allclose(Qh, Qg, atol=1e-15)
    assert np.allclose(dh[0], dg[1] + dg[4], atol=1e-14)


@pytest.mark.parametrize("which", ["hky", "gtr", "gy94"])
def test_rate_matrix_invariants(which):
    rng = np.random.default_rng(3)
    if which == "hky":
        pi = rng.dirichlet(np.ones(4))
        Q, dQ = model.hky(2.0, pi)
    elif which == "gtr":
        pi = rng.dirichlet(np.ones(4))
        Q, dQ = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)
    else:
        f = np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
        Q, pi, dQ = model.gy94(2.0, 0.3, f)
    S = len(pi)
    assert np.allclose(Q.sum(1), 0, atol=1e-13)
    assert abs(-np.dot(pi, np.diag(Q)) - 1.0) < 1e-13           # mean rate 1
    F = np.diag(pi) @ Q
    assert np.allclose(F, F.T, atol=1e-14)                        # reversibility
    for t in (0.0, 0.1, 1.0):
        P = expm(t * Q)
        assert np.allclose(P.sum(1), 1, atol=1e-13)
        if t == 0.0:
            assert np.allclose(P, np.eye(S), atol=1e-15)
        Fp = np.diag(pi) @ P
        assert np.allclose(Fp, Fp.T, atol=1e-14)                  # detailed balance
    Pinf = expm(5000.0 * Q)
    assert np.allclose(Pinf, np.outer(np.ones(S), pi), atol=1e-10)
    # eigen route (symmetrised Q) agrees with expm
    d = np.sqrt(pi)
    A = (d[:, None] * Q) / d[None, :]
    lam, U = np.linalg.eigh((A + A.T) / 2)
    for t in (0.05, 0.7):
        Pe = (U / d[:, None]) @ np.diag(np.exp(lam * t)) @ (U.T * d[None, :])
        assert np.allclose(Pe, expm(t * Q), atol=1e-13)
    # dQ/dtheta against central differences of the builder
    h = 1e-6
    for k, D in enumerate(dQ):
        if which == "hky":
            Qp, _ = model.hky(2.0 + h, pi); Qm, _ = model.hky(2.0 - h, pi)
        elif which == "gtr":
            r0 = rng.dirichlet(np.ones(6)) * 6
            Q0, dQ0 = model.gtr(r0, pi)
            rp, rm = r0.copy(), r0.copy(); rp[k] += h; rm[k] -= h
            Qp, _ = model.gtr(rp, pi); Qm, _ = model.gtr(rm, pi)
            D = dQ0[k]
        else:
            args = [2.0, 0.3]
            ap, am = list(args), list(args); ap[k] += h; am[k] -= h
            Qp = model.gy94(*ap, f)[0]; Qm = model.gy94(*am, f)[0]
        assert np.allclose((Qp - Qm) / (2 * h), D, atol=1e-8)


def test_gy94_structure():
    f = np.full((3, 4), 0.25)
    Q, pi, _ = model.gy94(1.0, 1.0, f)
    off = Q - np.diag(np.diag(Q))
    assert np.count_nonzero(off) == 526   # single-nucleotide sense-codon pairs
    # kappa = omega = 1 with uniform F3x4: every allowed change has one rate
    vals = off[off > 0]
    assert np.allclose(vals, vals[0])
    codons, amino = model.genetic_code()
    Q2, _, _ = model.gy94(1.0, 0.0, f)   # omega = 0 removes nonsynonymous changes
    for i in range(61):
        for j in range(61):
            if i != j and Q2[i, j] > 0:
                assert amino[i] == amino[j]


# ----------------------------------------------------------------------------
# likelihood
# ----------------------------------------------------------------------------

def test_two_taxon_jc_closed_form():
    tree = SimpleNamespace(n_tips=2, children=np.array([[0, 1]]),
                           edge_len=np.array([0.13, 0.29, 0.0]))
    pi = np.full(4, 0.25)
    Q, _ = model.hky(1.0, pi)
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = np.array([[0, 0, 1, 2, 3], [0, 1, 1, 3, 0]], dtype=np.int8)
    logl, site = pruning.loglik(tree, Q, pi, rates, cw, np.ones(5), states)
    d = 0.13 + 0.29
    want = []
    for a, b in states.T:
        L = 0.0
        for r, rho in enumerate(rates):
            e = np.exp(-4 * d * rho / 3)
            L += 0.25 * (0.25 * (0.25 + 0.75 * e) if a == b else 0.25 * (0.25 - 0.25 * e))
        want.append(np.log(L))
    assert np.allclose(site, want, rtol=1e-14, atol=0)
    assert abs(logl - sum(want)) < 1e-13 * abs(logl)


@pytest.mark.parametrize("n_tips,which,seed", [(2, "hky", 1), (3, "gtr", 2), (4, "hky", 3),
                                                (5, "gtr", 4), (6, "hky", 5), (6, "gtr", 6)])
@pytest.mark.parametrize("rescale", [True, False])
def test_pruning_equals_brute_force(n_tips, which, seed, rescale):
    rng = np.random.default_rng(seed)
    tree = small_tree(n_tips, seed)
    pi = rng.dirichlet(np.ones(4))
    Q = model.hky(2.0, pi)[0] if which == "hky" else model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = rng.dirichlet(np.ones(4))
    states = rand_states(rng, n_tips, 40, 4)
    logl, site = pruning.loglik(tree, Q, pi, rates, cw, np.ones(40), states, rescale)
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    L = brute.site_likelihood(tree.children, n_tips, P, pi, cw, pruning.tip_partials(states, 4))
    assert np.allclose(site, np.log(L), rtol=1e-13, atol=1e-13)


@pytest.mark.slow
def test_codon_pruning_equals_brute_force():
    rng = np.random.default_rng(11)
    tree = small_tree(3, 11)
    f = np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
    Q, pi, _ = model.gy94(2.0, 0.3, f)
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 3, 6, 61, 0.1)
    _, site = pruning.loglik(tree, Q, pi, rates, cw, np.ones(6), states)
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    L = brute.site_likelihood(tree.children, 3, P, pi, cw, pruning.tip_partials(states, 61))
    assert np.allclose(site, np.log(L), rtol=1e-12, atol=1e-12)


def test_root_placement_invariance_and_root_children_derivatives():
    rng = np.random.default_rng(7)
    tree = small_tree(9, 7)
    pi = rng.dirichlet(np.ones(4))
    Q = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 9, 50, 4)
    w = np.ones(50)
    base, _ = pruning.loglik(tree, Q, pi, rates, cw, w, states)
    for edge_child in (0, 3, 10, 12):
        for frac in (0.2, 0.5):
            t2 = reroot(tree, edge_child, frac)
            l2, _ = pruning.loglik(t2, Q, pi, rates, cw, w, states)
            assert abs(l2 - base) < 1e-12 * abs(base)
    g = gradient.branch_gradient(tree, Q, pi, rates, cw, w, states)
    a, b = tree.children[-1]
    assert abs(g[a] - g[b]) < 1e-10 * max(1.0, abs(g[a]))


def test_rescaling_and_weights():
    rng = np.random.default_rng(8)
    tree = small_tree(12, 8)
    pi = rng.dirichlet(np.ones(4))
    Q = model.hky(2.0, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 12, 30, 4)
    w = np.ones(30)
    l1, s1 = pruning.loglik(tree, Q, pi, rates, cw, w, states, rescale=True)
    l0, s0 = pruning.loglik(tree, Q, pi, rates, cw, w, states, rescale=False)
    assert abs(l1 - l0) < 1e-14 * abs(l0)
    # rescaled partial mantissas are bit-identical to the unscaled ones
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    tips = pruning.tip_partials(states, 4)
    ps, es = pruning.post_order(tree.children, 12, P, tips, True)
    pu, _ = pruning.post_order(tree.children, 12, P, tips, False)
    root = 22
    cum = sum(es.values())
    assert np.array_equal(np.frexp(ps[root])[0], np.frexp(pu[root])[0])
    assert np.array_equal(np.ldexp(ps[root], cum[None, :, None]), pu[root])
    # weight 2 == pattern duplicated; chunked == whole
    w2 = w.copy(); w2[5] = 2.0
    l2, _ = pruning.loglik(tree, Q, pi, rates, cw, w2, states)
    dup = np.concatenate([states, states[:, 5:6]], axis=1)
    l3, _ = pruning.loglik(tree, Q, pi, rates, cw, np.ones(31), dup)
    assert abs(l2 - l3) < 1e-13 * abs(l3)
    lc, _ = pruning.loglik_chunked(tree, Q, pi, rates, cw, w, states, chunk=7)
    assert abs(lc - l1) < 1e-12 * abs(l1)


def test_underflow_needs_rescaling():
    # a long caterpillar with long branches underflows FP64 without rescaling
    n = 700
    children = np.zeros((n - 1, 2), dtype=np.int64)
    children[0] = (0, 1)
    for k in range(1, n - 1):
        children[k] = (n + k - 1, k + 1)
    tree = SimpleNamespace(n_tips=n, children=children, edge_len=np.full(2 * n - 1, 3.0))
    pi = np.full(4, 0.25)
    Q = model.hky(1.0, pi)[0]
    rng = np.random.default_rng(1)
    states = rng.integers(0, 4, size=(n, 3)).astype(np.int8)
    l1, s1 = pruning.loglik(tree, Q, pi, np.ones(4), np.full(4, 0.25), np.ones(3), states)
    # near-saturated branches: each tip contributes about log(1/4)
    assert np.all(np.abs(s1 - n * np.log(0.25)) < 0.5)
    _, s0 = pruning.loglik(tree, Q, pi, np.ones(4), np.full(4, 0.25), np.ones(3), states,
                           rescale=False)
    assert np.all(np.isinf(s0))


# ----------------------------------------------------------------------------
# pre-order and gradients
# ----------------------------------------------------------------------------

def test_preorder_inner_product_is_likelihood_at_every_node():
    rng = np.random.default_rng(9)
    tree = small_tree(10, 9)
    pi = rng.dirichlet(np.ones(4))
    Q = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = rng.dirichlet(np.ones(4))
    states = rand_states(rng, 10, 25, 4)
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    tips = pruning.tip_partials(states, 4)
    post, exps = pruning.post_order(tree.children, 10, P, tips, rescale=False)
    q, u = gradient.pre_order(tree.children, 10, P, post, tips, pi, 4, rescale=False)
    _, site = pruning.loglik(tree, Q, pi, rates, cw, np.ones(25), states, rescale=False)
    L = np.exp(site)
    for v in range(2 * 10 - 2):
        pv = np.broadcast_to(tips[v], (4,) + tips[v].shape) if v < 10 else post[v]
        inner = np.einsum("r,rps,rps->p", cw, q[v], pv)
        assert np.allclose(inner, L, rtol=1e-13)


def _fd_branch(tree, v, h, f):
    t1 = SimpleNamespace(n_tips=tree.n_tips, children=tree.children, edge_len=tree.edge_len.copy())
    t2 = SimpleNamespace(n_tips=tree.n_tips, children=tree.children, edge_len=tree.edge_len.copy())
    t1.edge_len[v] += h
    t2.edge_len[v] -= h
    return (f(t1) - f(t2)) / (2 * h)


@pytest.mark.parametrize("which", ["hky", "gtr"])
def test_branch_gradient_vs_finite_differences(which):
    rng = np.random.default_rng(10)
    tree = small_tree(14, 10)
    pi = rng.dirichlet(np.ones(4))
    Q = model.hky(2.0, pi)[0] if which == "hky" else model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 14, 60, 4)
    w = rng.integers(1, 4, size=60).astype(float)
    g = gradient.branch_gradient(tree, Q, pi, rates, cw, w, states)
    f = lambda t: pruning.loglik(t, Q, pi, rates, cw, w, states)[0]
    for v in range(2 * 14 - 2):
        fd = _fd_branch(tree, v, 1e-6, f)
        assert abs(g[v] - fd) < 1e-6 * max(1.0, abs(fd)), (v, g[v], fd)
    assert g[tree.root if hasattr(tree, "root") else 26] == 0.0


def test_branch_gradient_vs_brute_force_derivative():
    rng = np.random.default_rng(12)
    tree = small_tree(5, 12)
    pi = rng.dirichlet(np.ones(4))
    Q = model.hky(3.0, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 5, 20, 4)
    w = np.ones(20)
    g = gradient.branch_gradient(tree, Q, pi, rates, cw, w, states)
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    tips = pruning.tip_partials(states, 4)
    L = brute.site_likelihood(tree.children, 5, P, pi, cw, tips)
    for v in range(8):
        Pd = P.copy()
        Pd[v] = np.einsum("r,ij,rjk->rik", rates, Q, P[v])   # d/dt expm(rho t Q)
        dL = brute.site_likelihood(tree.children, 5, Pd, pi, cw, tips)
        assert abs(g[v] - np.sum(dL / L)) < 1e-12 * max(1.0, abs(g[v]))


def test_substitution_gradient_vs_finite_differences():
    rng = np.random.default_rng(13)
    tree = small_tree(8, 13)
    pi = np.array([0.3, 0.2, 0.2, 0.3])
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 8, 40, 4)
    w = np.ones(40)
    Q, dQ = model.hky(2.0, pi)
    g = gradient.subst_gradient(tree, Q, dQ, pi, rates, cw, w, states)
    h = 1e-6
    lp = pruning.loglik(tree, model.hky(2.0 + h, pi)[0], pi, rates, cw, w, states)[0]
    lm = pruning.loglik(tree, model.hky(2.0 - h, pi)[0], pi, rates, cw, w, states)[0]
    assert abs(g[0] - (lp - lm) / (2 * h)) < 1e-6 * max(1, abs(g[0]))
    r0 = rng.dirichlet(np.ones(6)) * 6
    Q, dQ = model.gtr(r0, pi)
    g = gradient.subst_gradient(tree, Q, dQ, pi, rates, cw, w, states)
    for k in range(6):
        rp, rm = r0.copy(), r0.copy(); rp[k] += h; rm[k] -= h
        lp = pruning.loglik(tree, model.gtr(rp, pi)[0], pi, rates, cw, w, states)[0]
        lm = pruning.loglik(tree, model.gtr(rm, pi)[0], pi, rates, cw, w, states)[0]
        assert abs(g[k] - (lp - lm) / (2 * h)) < 1e-6 * max(1, abs(g[k]))


@pytest.mark.slow
def test_codon_gradients_vs_finite_differences():
    rng = np.random.default_rng(14)
    tree = small_tree(5, 14)
    f = np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
    Q, pi, dQ = model.gy94(2.0, 0.3, f)
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 5, 12, 61, 0.05)
    w = np.ones(12)
    g = gradient.subst_gradient(tree, Q, dQ, pi, rates, cw, w, states)
    h = 1e-6
    for k, (dk, dw) in enumerate(((h, 0), (0, h))):
        lp = pruning.loglik(tree, model.gy94(2.0 + dk, 0.3 + dw, f)[0], pi, rates, cw, w, states)[0]
        lm = pruning.loglik(tree, model.gy94(2.0 - dk, 0.3 - dw, f)[0], pi, rates, cw, w, states)[0]
        assert abs(g[k] - (lp - lm) / (2 * h)) < 1e-6 * max(1, abs(g[k]))
    gb = gradient.branch_gradient(tree, Q, pi, rates, cw, w, states)
    fl = lambda t: pruning.loglik(t, Q, pi, rates, cw, w, states)[0]
    for v in (0, 3, 6):
        fd = _fd_branch(tree, v, 1e-6, fl)
        assert abs(gb[v] - fd) < 1e-6 * max(1.0, abs(fd))


# ----------------------------------------------------------------------------
# dlogL/dP per edge and dlogL/dQ (the reverse-mode substitution gradient)
# ----------------------------------------------------------------------------

def test_edge_adjoints_vs_brute_force_derivative():
    """M[v, r][i, j] = dlogL/dP_r(t_v)[i, j]: the likelihood by enumeration is
    linear in each matrix entry, so the derivative is exact from one
    perturbed evaluation; also sum_r <M[v, r], rho_r Q P> = dlogL/dt_v."""
    rng = np.random.default_rng(31)
    tree = small_tree(4, 31)
    pi = rng.dirichlet(np.ones(4))
    Q = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5, 3)
    cw = np.array([0.2, 0.5, 0.3])
    states = rand_states(rng, 4, 25, 4)
    w = rng.integers(1, 4, size=25).astype(float)
    M = gradient.edge_adjoints(tree, Q, pi, rates, cw, w, states)
    P = pruning.transition_matrices(Q, tree.edge_len, rates)
    tips = pruning.tip_partials(states, 4)
    L = brute.site_likelihood(tree.children, 4, P, pi, cw, tips)
    for v in (0, 2, 4, 5):
        for r in range(3):
            for i, j in ((0, 0), (1, 3), (3, 2)):
                E = np.zeros_like(P)
                E[v, r, i, j] = 1.0
                # L is linear in P[v, r]: the derivative is L(E-only) (the
                # other matrices unchanged, this one replaced by E)
                Pd = P.copy()
                Pd[v] = 0.0
                Pd[v, r] = E[v, r]
                dL = brute.site_likelihood(tree.children, 4, Pd, pi, cw, tips)
                assert abs(M[v, r, i, j] - np.dot(w, dL / L)) < 1e-11 * max(1, abs(M[v, r, i, j]))
    g = gradient.branch_gradient(tree, Q, pi, rates, cw, w, states)
    for v in range(6):
        gv = sum(rates[r] * np.sum(M[v, r] * (Q @ P[v, r])) for r in range(3))
        assert abs(gv - g[v]) < 1e-11 * max(1, abs(g[v]))


def test_rate_matrix_gradient_vs_finite_differences():
    """dlogL/dQ against central differences of logL in single entries of Q,
    diagonal and off-diagonal, including directions that break
    reversibility (expm of any Q is defined)."""
    rng = np.random.default_rng(32)
    tree = small_tree(7, 32)
    pi = rng.dirichlet(np.ones(4))
    Q = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 7, 50, 4)
    w = rng.integers(1, 3, size=50).astype(float)
    G = gradient.rate_matrix_gradient(tree, Q, pi, rates, cw, w, states)
    h = 1e-6
    for i, j in ((0, 1), (1, 0), (2, 2), (3, 1), (0, 3)):
        Qp, Qm = Q.copy(), Q.copy()
        Qp[i, j] += h
        Qm[i, j] -= h
        fd = (pruning.loglik(tree, Qp, pi, rates, cw, w, states)[0]
              - pruning.loglik(tree, Qm, pi, rates, cw, w, states)[0]) / (2 * h)
        assert abs(G[i, j] - fd) < 1e-6 * max(1, abs(fd)), (i, j, G[i, j], fd)


def test_rate_matrix_gradient_euler_identity_and_first_order():
    """Scaling Q by (1 + e) is scaling every branch length by (1 + e), so
    <dlogL/dQ, Q> = sum_v t_v dlogL/dt_v. The first-order approximation is
    exact in any direction that commutes with Q (Q itself; dQ/dkappa of HKY,
    whose eigenvectors do not depend on kappa) and not in general."""
    rng = np.random.default_rng(33)
    tree = small_tree(9, 33)
    pi = rng.dirichlet(np.ones(4))
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, 9, 40, 4)
    w = np.ones(40)
    Q, dQ = model.hky(3.0, pi)
    args = (tree, Q, pi, rates, cw, w, states)
    G = gradient.rate_matrix_gradient(*args)
    Ga = gradient.rate_matrix_gradient(*args, first_order=True)
    g = gradient.branch_gradient(*args)
    ref = np.dot(tree.edge_len[:16], g[:16])
    assert abs(np.sum(G * Q) - ref) < 1e-10 * abs(ref)
    assert abs(np.sum(Ga * Q) - ref) < 1e-10 * abs(ref)
    gk = gradient.subst_gradient(tree, Q, dQ, pi, rates, cw, w, states)[0]
    assert abs(np.sum(G * dQ[0]) - gk) < 1e-10 * max(1, abs(gk))
    assert abs(np.sum(Ga * dQ[0]) - gk) < 1e-10 * max(1, abs(gk))
    Q2, dQ2 = model.gtr(rng.dirichlet(np.ones(6)) * 6, pi)
    G2 = gradient.rate_matrix_gradient(tree, Q2, pi, rates, cw, w, states)
    Ga2 = gradient.rate_matrix_gradient(tree, Q2, pi, rates, cw, w, states, first_order=True)
    assert np.max(np.abs(G2 - Ga2)) > 1e-3 * np.max(np.abs(G2))


def test_complex_step_jacobian_matches_hand_derivatives():
    f = np.stack([np.random.default_rng(34 + k).dirichlet(np.ones(4)) for k in range(3)])
    pi4 = np.array([0.1, 0.2, 0.3, 0.4])
    for name, params, freqs in (("hky", [2.5], pi4), ("gtr", [1, 2, 0.5, 0.7, 3, 1], pi4),
                                ("gy94", [2.0, 0.3], f)):
        J = model.rate_jacobian(name, params, freqs)
        D = np.array(model.build(name, params, freqs)[2])
        assert np.max(np.abs(J - D)) < 1e-13 * np.max(np.abs(D))
    # random effects: Q(eps) by central differences of the builder
    eps = np.random.default_rng(35).normal(0, 0.3, 263)
    p0 = np.r_[2.0, 0.3, eps]
    J = model.rate_jacobian("gy94re", p0, f)
    for k in (2, 50, 264):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += 1e-6
        pm[k] -= 1e-6
        fd = (model.build("gy94re", pp, f)[0] - model.build("gy94re", pm, f)[0]) / 2e-6
        assert np.max(np.abs(J[k] - fd)) < 1e-8   # entries of Q are O(1)
        assert np.max(np.abs(J[k])) > 1e-5
    Q0 = model.build("gy94re", np.r_[2.0, 0.3, np.zeros(263)], f)[0]
    assert np.array_equal(Q0, model.gy94(2.0, 0.3, f)[0])
    assert len(model.gy94_pairs()) == 263


@pytest.mark.slow
def test_random_effects_gradient_vs_finite_differences():
    """dlogL/deps_k = <dlogL/dQ, dQ/deps_k> against central differences of
    logL through the random-effects GY94 builder (3 taxa, 61 states)."""
    rng = np.random.default_rng(36)
    tree = small_tree(3, 36)
    f = np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
    eps = rng.normal(0, 0.3, 263)
    p0 = np.r_[2.0, 0.3, eps]
    Q, pi, _ = model.build("gy94re", p0, f)
    rates = synth.gamma_rates(0.5, 2)
    cw = np.full(2, 0.5)
    states = rand_states(rng, 3, 10, 61, 0.0)
    w = np.ones(10)
    G = gradient.rate_matrix_gradient(tree, Q, pi, rates, cw, w, states)
    J = model.rate_jacobian("gy94re", p0, f)
    h = 1e-6
    for k in (0, 1, 2, 77, 264):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        fd = (pruning.loglik(tree, model.build("gy94re", pp, f)[0], pi, rates, cw, w, states)[0]
              - pruning.loglik(tree, model.build("gy94re", pm, f)[0], pi, rates, cw, w, states)[0]) / (2 * h)
        assert abs(np.sum(G * J[k]) - fd) < 1e-6 * max(1, abs(fd)), (k, np.sum(G * J[k]), fd)


def test_general_reversible_model_pins():
    """The general reversible model with GTR's exchangeabilities is GTR; on
    20 states its Q has zero row sums, unit mean rate and detailed balance."""
    g = [1.0, 2.0, 0.5, 0.7, 3.0, 1.2]
    pi4 = np.array([0.1, 0.2, 0.3, 0.4])
    E = np.zeros((4, 4))
    for k, (i, j) in enumerate(model.GTR_PAIRS):
        E[i, j] = E[j, i] = g[k]
    assert np.allclose(model.rev(E, pi4), model.gtr(g, pi4)[0], rtol=1e-15, atol=1e-15)
    w = synth.workload("aa20_256x10k", n_tips=5, n_patterns=20)
    Q, pi, dQ = model.build("rev", w.params, w.freqs)
    assert Q.shape == (20, 20) and dQ == []
    assert np.max(np.abs(Q.sum(axis=1))) < 1e-14
    assert abs(-np.dot(pi, np.diag(Q)) - 1.0) < 1e-14
    D = pi[:, None] * Q
    assert np.max(np.abs(D - D.T)) < 1e-16


def test_ratio_transform_chain_rule_vs_finite_differences():
    """Ratios, root height and branch rates: the chain rule against central
    differences of logL through the transform (tips at different heights)."""
    from oracle import ratio
    rng = np.random.default_rng(41)
    tree = small_tree(9, 41)
    n = 9
    tip_h = rng.uniform(0.0, 0.3, n)
    r = rng.uniform(0.2, 0.8, n - 1)
    root_h = 1.5
    rate = rng.uniform(0.5, 1.5, 2 * n - 1)
    pi = rng.dirichlet(np.ones(4))
    Q = model.hky(2.0, pi)[0]
    rates = synth.gamma_rates(0.5)
    cw = np.full(4, 0.25)
    states = rand_states(rng, n, 40, 4)
    w = np.ones(40)

    def f(rr, rh, rt):
        h = ratio.heights(tree.children, n, tip_h, rr, rh)
        assert np.all(h[n:] > ratio.anchors(tree.children, n, tip_h)[n:])
        t = ratio.branch_lengths(tree.children, n, h, rt)
        tr = SimpleNamespace(n_tips=n, children=tree.children, edge_len=t)
        return pruning.loglik(tr, Q, pi, rates, cw, w, states)[0]

    h = ratio.heights(tree.children, n, tip_h, r, root_h)
    t = ratio.branch_lengths(tree.children, n, h, rate)
    tr = SimpleNamespace(n_tips=n, children=tree.children, edge_len=t)
    g = gradient.branch_gradient(tr, Q, pi, rates, cw, w, states)
    gr, grh, grate = ratio.ratio_gradient(tree.children, n, tip_h, r, root_h, rate, g)
    eps = 1e-6
    for k in range(n - 2):
        rp, rm = r.copy(), r.copy()
        rp[k] += eps
        rm[k] -= eps
        fd = (f(rp, root_h, rate) - f(rm, root_h, rate)) / (2 * eps)
        assert abs(gr[k] - fd) < 1e-6 * max(1.0, abs(fd)), (k, gr[k], fd)
    fd = (f(r, root_h + eps, rate) - f(r, root_h - eps, rate)) / (2 * eps)
    assert abs(grh - fd) < 1e-6 * max(1.0, abs(fd))
    for v in (0, 5, 12):
        pp, pm = rate.copy(), rate.copy()
        pp[v] += eps
        pm[v] -= eps
        fd = (f(r, root_h, pp) - f(r, root_h, pm)) / (2 * eps)
        assert abs(grate[v] - fd) < 1e-6 * max(1.0, abs(fd))


def _f3x4_worked():
    """The hand-worked F3x4 example of tests/golden/f3x4_worked.txt."""
    f, rows = [], []
    with open(os.path.join(GOLDEN, "f3x4_worked.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if not line:
                continue
            if line[0] in ("f1", "f2", "f3"):
                f.append([float(x) for x in line[1:]])
            else:
                rows.append((line[0], int(line[1]), float(line[2])))
    return np.array(f), rows


def test_f3x4_frequencies_match_the_worked_example():
    """Non-uniform position frequencies, so a position mix-up (f1 used at
    every position, positions swapped) or a missing stop renormalisation
    changes the pinned values."""
    f, rows = _f3x4_worked()
    pi = model.f3x4_frequencies(f)
    codons, _ = model.genetic_code()
    assert len(pi) == 61 and abs(pi.sum() - 1.0) < 1e-15
    for name, idx, num in rows:
        assert "".join(model.BASES[b] for b in codons[idx]) == name
        assert abs(pi[idx] - num / 0.908) <= 1e-15, (name, pi[idx], num / 0.908)


def test_gy94_rate_ratios_on_the_worked_frequencies():
    """Off-diagonal GY94 rates out of one codon are kappa^[ts] omega^[ns] pi_j
    up to the common normaliser: AAA (Lys) -> AAG (Lys) is a synonymous
    transition, AAA -> AAC (Asn) a nonsynonymous transversion, AAA -> GAA
    (Glu) a nonsynonymous transition, AAA -> AAT (Asn) a nonsynonymous
    transversion; AAA -> ACC (two changes) has rate zero."""
    f, rows = _f3x4_worked()
    kappa, omega = 2.5, 0.3
    Q, pi, _ = model.gy94(kappa, omega, f)
    idx = {"".join(model.BASES[b] for b in c): i for i, c in enumerate(model.genetic_code()[0])}
    # pi by hand: AAG = .1*.4*.2, AAC = .1*.4*.15, GAA = .3*.4*.25, AAT = .1*.4*.4 (over .908)
    q = lambda a, b: Q[idx[a], idx[b]]
    assert abs(q("AAA", "AAG") / q("AAA", "AAC") - (kappa * 0.008) / (omega * 0.006)) < 1e-12
    assert abs(q("AAA", "GAA") / q("AAA", "AAT") - (kappa * omega * 0.030) / (omega * 0.016)) < 1e-12
    assert q("AAA", "ACC") == 0.0
