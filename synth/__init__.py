"""Seeded synthetic inputs for the phylogenetic likelihood path.

This module is the only code that both the FP64 oracle tests and the CUDA
library's tests and benchmark use. It draws trees, branch lengths, model
parameters and alignments; it holds none of the likelihood method's
arithmetic (no rate matrix of HKY, GTR or GY94, no matrix exponential, no
pruning). Alignments are simulated down the tree with the equal-input jump
process of Felsenstein (1981): along a branch of length t in rate category
rho a site keeps its state with probability exp(-beta*rho*t) and otherwise
redraws it from the stationary frequencies, beta normalising the expected
substitution rate to one. Codon stationary draws are three nucleotide draws
from per-position frequencies, redrawn while they spell a stop codon.

Workload shapes follow the paper's benchmarks (Sec. "Performance
evaluation": HKY and GY94 on fixed trees with up to 1,024 taxa, patterns
1 to 2,048; GTR on 352 taxa x 2,294 patterns); sizes are those of the
synthetic configurations named in ``CONFIGS``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import special

ROOT_SEED = 20261203
NUC = "ACGT"
# The three stop codons of the standard genetic code (TAA, TAG, TGA) are the
# only codons a simulated site may never hold.
_STOPS = {(3, 0, 0), (3, 0, 2), (3, 2, 0)}


def _sense_codon_index():
    """Map (n1, n2, n3) nucleotide triples to 0..60, lexicographic in ACGT."""
    idx = {}
    k = 0
    for a in range(4):
        for b in range(4):
            for c in range(4):
                if (a, b, c) in _STOPS:
                    continue
                idx[(a, b, c)] = k
                k += 1
    return idx


_CODON_INDEX = _sense_codon_index()


def rng_for(config: int, stream: str) -> np.random.Generator:
    """PCG64 generator for substream ``stream`` of configuration ``config``.

    SeedSequence(ROOT_SEED).spawn gives one child per configuration; each
    configuration spawns fixed substreams for tree, params and sites.
    """
    names = ("tree", "params", "sites", "extra")
    root = np.random.SeedSequence(ROOT_SEED)
    child = root.spawn(config + 1)[config]
    sub = child.spawn(len(names))[names.index(stream)]
    return np.random.Generator(np.random.PCG64(sub))


@dataclass
class Tree:
    """Rooted binary tree.

    Tips are 0..n_tips-1; internal nodes n_tips..2*n_tips-2 are numbered in
    post-order (both children of a node have smaller indices) so the root is
    2*n_tips-2. ``children[k]`` are the two children of internal node
    n_tips+k; ``edge_len[v]`` is the length of the edge above node v
    (0 for the root); ``parent[root] = -1``.
    """

    n_tips: int
    children: np.ndarray
    parent: np.ndarray
    edge_len: np.ndarray

    @property
    def root(self) -> int:
        return 2 * self.n_tips - 2

    @property
    def n_nodes(self) -> int:
        return 2 * self.n_tips - 1


def yule_topology(n_tips: int, rng: np.random.Generator) -> Tree:
    """Yule (pure-birth) topology: start from a root with two leaves and split
    a uniformly chosen leaf until there are ``n_tips`` leaves."""
    if n_tips < 2:
        raise ValueError("need at least two tips")
    kids = {0: [1, 2]}
    leaves = [1, 2]
    nxt = 3
    while len(leaves) < n_tips:
        j = int(rng.integers(len(leaves)))
        v = leaves[j]
        kids[v] = [nxt, nxt + 1]
        leaves[j] = nxt
        leaves.append(nxt + 1)
        nxt += 2
    # relabel: leaves in a random order become tips 0..n-1, internal nodes get
    # post-order labels n..2n-2
    perm = rng.permutation(len(leaves))
    label = {}
    for t, li in enumerate(perm):
        label[leaves[li]] = t
    order = []
    stack = [(0, False)]
    while stack:
        v, done = stack.pop()
        if v not in kids:
            continue
        if done:
            order.append(v)
        else:
            stack.append((v, True))
            stack.append((kids[v][1], False))
            stack.append((kids[v][0], False))
    for k, v in enumerate(order):
        label[v] = n_tips + k
    children = np.zeros((n_tips - 1, 2), dtype=np.int64)
    parent = -np.ones(2 * n_tips - 1, dtype=np.int64)
    for v, (a, b) in kids.items():
        children[label[v] - n_tips] = (label[a], label[b])
        parent[label[a]] = label[v]
        parent[label[b]] = label[v]
    return Tree(n_tips, children, parent, np.zeros(2 * n_tips - 1))


def yule_tree(n_tips: int, rng: np.random.Generator, mean_len: float = 0.1) -> Tree:
    """Yule topology with i.i.d. Exp(mean ``mean_len``) branch lengths."""
    t = yule_topology(n_tips, rng)
    el = rng.exponential(mean_len, size=2 * n_tips - 1)
    el[t.root] = 0.0
    t.edge_len = el
    return t


def gamma_rates(alpha: float, ncat: int = 4) -> np.ndarray:
    """Discrete-Gamma category rates by Yang's (1994) mean method: the
    Gamma(alpha, alpha) density is cut into ``ncat`` equal-probability bins
    and each category takes the mean of its bin (rates average to 1)."""
    cuts = special.gammaincinv(alpha, np.arange(1, ncat) / ncat) / alpha
    # mean of Gamma(a, a) over [lo, hi) times ncat uses the Gamma(a+1, a) cdf
    upper = np.concatenate([special.gammainc(alpha + 1, cuts * alpha), [1.0]])
    lower = np.concatenate([[0.0], upper[:-1]])
    return (upper - lower) * ncat


def _f81_down(tree: Tree, n_sites: int, n_states: int, cats: np.ndarray,
              rates: np.ndarray, beta: float, draw, rng, sparse: bool = False) -> np.ndarray:
    states = np.empty((tree.n_nodes, n_sites), dtype=np.int64)
    states[tree.root] = draw(n_sites)
    # walk parents before children: internal labels are post-order, so a
    # decreasing sweep over internal nodes reaches parents first
    for node in range(tree.root, tree.n_tips - 1, -1):
        a, b = tree.children[node - tree.n_tips]
        for c in (a, b):
            keep = np.exp(-beta * rates[cats] * tree.edge_len[c])
            u = rng.random(n_sites)
            if sparse:
                # the same process, drawing new states only where a jump happens
                states[c] = states[node]
                jump = np.nonzero(u >= keep)[0]
                states[c, jump] = draw(jump.size)
            else:
                new = draw(n_sites)
                states[c] = np.where(u < keep, states[node], new)
    return states[: tree.n_tips]


def simulate_nucleotide(tree: Tree, pi: np.ndarray, rates: np.ndarray,
                        n_sites: int, rng: np.random.Generator,
                        sparse: bool = False) -> np.ndarray:
    """int8 [n_tips, n_sites] nucleotide states (0..3 = A,C,G,T)."""
    pi = np.asarray(pi, dtype=float)
    beta = 1.0 / (1.0 - float(np.sum(pi * pi)))
    cats = rng.integers(len(rates), size=n_sites)

    def draw(n):
        return rng.choice(4, size=n, p=pi)

    return _f81_down(tree, n_sites, 4, cats, np.asarray(rates), beta, draw,
                     rng, sparse).astype(np.int8)


def simulate_states(tree: Tree, pi: np.ndarray, rates: np.ndarray, n_sites: int,
                    rng: np.random.Generator) -> np.ndarray:
    """int8 [n_tips, n_sites] states 0..S-1 (S = len(pi)) under the
    equal-input jump process with stationary pi (amino acids: S = 20)."""
    pi = np.asarray(pi, dtype=float)
    beta = 1.0 / (1.0 - float(np.sum(pi * pi)))
    cats = rng.integers(len(rates), size=n_sites)

    def draw(n):
        return rng.choice(len(pi), size=n, p=pi)

    return _f81_down(tree, n_sites, len(pi), cats, np.asarray(rates), beta, draw,
                     rng).astype(np.int8)


def simulate_codon(tree: Tree, f3x4: np.ndarray, rates: np.ndarray,
                   n_sites: int, rng: np.random.Generator, sparse: bool = False) -> np.ndarray:
    """int8 [n_tips, n_sites] sense-codon states (0..60, ACGT-lexicographic
    with TAA, TAG, TGA removed). ``f3x4`` is [3, 4] per-position nucleotide
    frequencies; a stationary draw takes one nucleotide per position and is
    redrawn while it spells a stop codon."""
    f3x4 = np.asarray(f3x4, dtype=float)
    lut = -np.ones(64, dtype=np.int64)
    for (a, b, c), k in _CODON_INDEX.items():
        lut[16 * a + 4 * b + c] = k

    def draw(n):
        out = np.empty(n, dtype=np.int64)
        todo = np.arange(n)
        while todo.size:
            code = (16 * rng.choice(4, size=todo.size, p=f3x4[0])
                    + 4 * rng.choice(4, size=todo.size, p=f3x4[1])
                    + rng.choice(4, size=todo.size, p=f3x4[2]))
            k = lut[code]
            ok = k >= 0
            out[todo[ok]] = k[ok]
            todo = todo[~ok]
        return out

    # expected-rate normaliser of the equal-input process: one over the
    # probability that a stationary redraw lands on a different codon
    w = np.array([f3x4[0, a] * f3x4[1, b] * f3x4[2, c]
                  for (a, b, c) in _CODON_INDEX])
    w /= w.sum()
    beta = 1.0 / (1.0 - float(np.sum(w * w)))
    cats = rng.integers(len(rates), size=n_sites)
    return _f81_down(tree, n_sites, 61, cats, np.asarray(rates), beta, draw,
                     rng, sparse).astype(np.int8)


@dataclass
class Workload:
    """One synthetic problem: tree, model parameters and alignment.

    ``model`` is "hky", "gtr" or "gy94"; ``params`` holds kappa (hky),
    the six exchangeabilities AC,AG,AT,CG,CT,GT (gtr), or kappa, omega (gy94);
    ``freqs`` is pi (4 values) for nucleotides or the [3, 4] F3x4 position
    frequencies for gy94. ``tips`` is int8 [n_tips, n_patterns].
    """

    name: str
    tree: Tree
    model: str
    params: np.ndarray
    freqs: np.ndarray
    alpha: float
    rates: np.ndarray
    cat_weights: np.ndarray
    pattern_weights: np.ndarray
    tips: np.ndarray
    n_states: int
    extra: dict = field(default_factory=dict)

    @property
    def n_patterns(self) -> int:
        return int(self.tips.shape[1])


def make_workload(config: int, *, model: str, n_tips: int, n_patterns: int,
                  alpha: float = 0.5, kappa: float = 2.0, omega: float = 0.3,
                  pi=None, name: str | None = None, n_states: int = 20) -> Workload:
    """Draw a workload from configuration ``config``'s seed streams."""
    rt, rp, rs = rng_for(config, "tree"), rng_for(config, "params"), rng_for(config, "sites")
    tree = yule_tree(n_tips, rt)
    rates = gamma_rates(alpha, 4)
    cw = np.full(4, 0.25)
    if model == "hky":
        freqs = np.asarray(pi if pi is not None else rp.dirichlet(np.ones(4)), float)
        params = np.array([kappa])
        tips = simulate_nucleotide(tree, freqs, rates, n_patterns, rs)
        S = 4
    elif model == "gtr":
        params = rp.dirichlet(np.ones(6)) * 6.0
        freqs = np.asarray(pi if pi is not None else rp.dirichlet(np.ones(4)), float)
        tips = simulate_nucleotide(tree, freqs, rates, n_patterns, rs)
        S = 4
    elif model == "gy94":
        params = np.array([kappa, omega])
        freqs = np.stack([rp.dirichlet(np.ones(4)) for _ in range(3)])
        tips = simulate_codon(tree, freqs, rates, n_patterns, rs)
        S = 61
    elif model == "rev":
        # amino acids: symmetric exchangeabilities ~ Exp(1) (row-major S x S,
        # mirrored), frequencies ~ Dirichlet(1)
        S = n_states
        e = rp.exponential(1.0, size=(S, S))
        params = np.triu(e, 1) + np.triu(e, 1).T
        freqs = rp.dirichlet(np.ones(S))
        tips = simulate_states(tree, freqs, rates, n_patterns, rs)
    else:
        raise ValueError(model)
    return Workload(name or f"config{config}", tree, model, params, freqs, alpha,
                    rates, cw, np.ones(n_patterns), tips, S)


# The five workloads the measurements are quoted on (names give their shape).
CONFIGS = {
    "hky_8x1000": dict(config=0, model="hky", n_tips=8, n_patterns=1000,
                       pi=[0.3, 0.2, 0.2, 0.3], kappa=2.0),
    "gtr_512x100k": dict(config=1, model="gtr", n_tips=512, n_patterns=100_000),
    "gy94_128x20k": dict(config=2, model="gy94", n_tips=128, n_patterns=20_000,
                         kappa=2.0, omega=0.3),
    "gtr_1024x50k": dict(config=3, model="gtr", n_tips=1024, n_patterns=50_000),
    "gy94_64x5k": dict(config=3, model="gy94", n_tips=64, n_patterns=5_000,
                       kappa=2.0, omega=0.3),
    # amino acids (20 states, a general reversible model): a "next" workload
    "aa20_256x10k": dict(config=5, model="rev", n_tips=256, n_patterns=10_000, n_states=20),
    # phylogeography: 64 discrete locations, one site pattern
    "geo64_1024x1": dict(config=6, model="rev", n_tips=1024, n_patterns=1, n_states=64),
}


def workload(name: str, **override) -> Workload:
    kw = dict(CONFIGS[name])
    kw.update(override)
    return make_workload(name=name, **kw)


N_GY94_PAIRS = 263   # codon pairs one nucleotide apart (the non-zero rates)


def random_effects(config: int = 3, sd: float = 0.3) -> np.ndarray:
    """One log-scale random effect per non-zero GY94 off-diagonal pair,
    i.i.d. Normal(0, sd), from the configuration's "extra" substream."""
    return rng_for(config, "extra").normal(0.0, sd, N_GY94_PAIRS)


# ---------------------------------------------------------------------------
# serving stream: requests from many MCMC chains
# ---------------------------------------------------------------------------
SERVING_CONFIG = 4


@dataclass
class ServingRequest:
    """One likelihood (or likelihood + gradient) request of a chain: a tree
    proposal (new branch lengths on the chain's topology) and the chain's
    current substitution-model parameters, so a request alone fixes its
    result."""

    chain: int
    edge_len: np.ndarray
    params: np.ndarray
    gradient: bool


def _loguniform_int(rng, lo: int, hi: int) -> int:
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def _chunked(sim, tree, freqs, rates, n_sites, rng, chunk=16384) -> np.ndarray:
    """Simulate in site chunks so memory stays O(nodes x chunk)."""
    parts = [sim(tree, freqs, rates, min(chunk, n_sites - s), rng, sparse=True)
             for s in range(0, n_sites, chunk)]
    return np.concatenate(parts, axis=1)


def serving_stream(n_requests: int = 2000, n_chains: int = 128, *, taxa=(16, 1024),
                   patterns=(100, 200_000), codon_frac: float = 0.3, grad_frac: float = 0.5,
                   param_move_frac: float = 0.2, alpha: float = 0.5):
    """(chains, requests, gaps) of the serving workload.

    Chains draw taxa and pattern counts log-uniformly in the given ranges;
    a chain is GY94 codon with probability ``codon_frac``, otherwise HKY or
    GTR with equal probability. Every request picks a chain uniformly, keeps
    its topology and multiplies each branch length by a log-normal factor
    (sd 0.1); with probability ``param_move_frac`` the chain's model
    parameters take a log-normal step (sd 0.1) first; with probability
    ``grad_frac`` it asks for the gradient as well. ``gaps`` are unit-mean exponential inter-arrival times
    (a Poisson process, scaled to the offered load by the caller)."""
    root = np.random.SeedSequence(ROOT_SEED).spawn(SERVING_CONFIG + 1)[SERVING_CONFIG]
    s_chain, s_req = root.spawn(2)
    rq = np.random.Generator(np.random.PCG64(s_req))
    chains = []
    for c, ss in enumerate(s_chain.spawn(n_chains)):
        rng = np.random.Generator(np.random.PCG64(ss))
        n_tips = max(2, _loguniform_int(rng, *taxa))
        n_pat = max(1, _loguniform_int(rng, *patterns))
        u = rng.random()
        model = "gy94" if u < codon_frac else ("hky" if u < codon_frac + (1 - codon_frac) / 2
                                               else "gtr")
        tree = yule_tree(n_tips, rng)
        rates = gamma_rates(alpha, 4)
        if model == "hky":
            freqs = rng.dirichlet(np.ones(4))
            params = np.array([2.0])
            tips = _chunked(simulate_nucleotide, tree, freqs, rates, n_pat, rng)
            S = 4
        elif model == "gtr":
            params = rng.dirichlet(np.ones(6)) * 6.0
            freqs = rng.dirichlet(np.ones(4))
            tips = _chunked(simulate_nucleotide, tree, freqs, rates, n_pat, rng)
            S = 4
        else:
            params = np.array([2.0, 0.3])
            freqs = np.stack([rng.dirichlet(np.ones(4)) for _ in range(3)])
            tips = _chunked(simulate_codon, tree, freqs, rates, n_pat, rng)
            S = 61
        chains.append(Workload(f"chain{c}", tree, model, params, freqs, alpha, rates,
                               np.full(4, 0.25), np.ones(n_pat), tips, S))
    requests = []
    current = [np.asarray(w.params, dtype=float).copy() for w in chains]
    for _ in range(n_requests):
        c = int(rq.integers(n_chains))
        w = chains[c]
        el = w.tree.edge_len * np.exp(rq.normal(0.0, 0.1, size=w.tree.edge_len.size))
        el[w.tree.root] = 0.0
        if rq.random() < param_move_frac:
            current[c] = current[c] * np.exp(rq.normal(0.0, 0.1, size=current[c].size))
        requests.append(ServingRequest(c, el, current[c].copy(), bool(rq.random() < grad_frac)))
    gaps = rq.exponential(1.0, size=n_requests)
    return chains, requests, gaps
