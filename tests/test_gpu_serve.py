"""Continuous-batching server: each request's result is the same alone and in
the mix (bit-identical: four-state requests share batched launches whose
per-instance arithmetic does not depend on the batch, codon requests run
their own passes), matches the FP64 oracle, and survives admission under a
memory budget small enough to force evictions, checkpointed service of a
chain too large for its whole-tree buffers, and a rejection."""
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


@pytest.fixture(scope="module")
def stream():
    # small chains: 4 to 40 taxa, 10 to 3,000 patterns, 30% codon
    return synth.serving_stream(60, 8, taxa=(4, 40), patterns=(10, 3000))


def serve(chains, reqs, budget=None, arrivals=None):
    from paper_2606_27607_gb300.serve import Server, run_open_loop
    s = Server(memory_budget=budget)
    for w in chains:
        s.add_chain(w)
    try:
        if arrivals is None:
            futs = [s.submit(r) for r in reqs]
            s.drain()
        else:
            futs, _ = run_open_loop(s, reqs, arrivals)
        out = []
        for f in futs:
            e = f.exception()
            out.append(e if e is not None else f.result())
        return out, dict(s.stats), list(s.group_sizes)
    finally:
        s.close()


def test_same_alone_and_in_the_mix(stream):
    chains, reqs, gaps = stream
    mixed, stats, sizes = serve(chains, reqs)
    assert max(sizes) > 1          # requests really shared launches
    for i in range(0, len(reqs), 7):
        alone, _, _ = serve(chains, reqs[i:i + 1])
        a, m = alone[0], mixed[i]
        assert a.logl == m.logl, i
        if reqs[i].gradient:
            assert np.array_equal(a.gradient, m.gradient), i
        else:
            assert a.gradient is None and m.gradient is None


def test_open_loop_arrivals_give_same_results(stream):
    chains, reqs, gaps = stream
    base, _, _ = serve(chains, reqs)
    arrivals = np.cumsum(gaps) * 2e-3      # about 500 requests/s offered
    got, _, _ = serve(chains, reqs, arrivals=arrivals)
    for a, b in zip(base, got):
        assert a.logl == b.logl
        assert (a.gradient is None) == (b.gradient is None)
        if a.gradient is not None:
            assert np.array_equal(a.gradient, b.gradient)
        assert b.latency > 0


def test_results_match_oracle(stream):
    chains, reqs, _ = stream
    got, _, _ = serve(chains, reqs[:12])
    for i, (r, g) in enumerate(zip(reqs[:12], got)):
        w = chains[r.chain]
        Q, pi, _ = om.build(w.model, r.params, w.freqs)
        tree = synth.Tree(w.tree.n_tips, w.tree.children, w.tree.parent, r.edge_len)
        want, _ = op.loglik(tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
        assert abs(g.logl - want) <= 1e-5 * abs(want), (r.chain, g.logl, want)
        if r.gradient:
            wg = og.branch_gradient(tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                    w.tips)
            scale = np.max(np.abs(wg))
            assert np.max(np.abs(g.gradient - wg) / np.maximum(np.abs(wg), 1e-3 * scale)) <= 1e-3


def test_admission_under_a_small_budget(stream):
    from paper_2606_27607_gb300.serve import footprint
    chains, reqs, _ = stream
    base, _, _ = serve(chains, reqs)
    sizes = sorted(footprint(w.tree.n_tips, w.n_patterns, w.n_states,
                             "f32" if w.n_states == 4 else "tf32x3") for w in chains)
    # room for the largest chain but not for all of them at once
    budget = sizes[-1] + sizes[-2] // 2
    got, stats, _ = serve(chains, reqs, budget=budget)
    assert stats.get("evicted", 0) > 0
    for a, b in zip(base, got):
        assert a.logl == b.logl
    # a budget below the largest chain's whole-tree buffers serves it with
    # subtree checkpointing, with bit-identical results
    from paper_2606_27607_gb300.checkpoint import best_band
    big = max(range(len(chains)), key=lambda k: footprint(
        chains[k].tree.n_tips, chains[k].n_patterns, chains[k].n_states,
        "f32" if chains[k].n_states == 4 else "tf32x3"))
    got, stats, _ = serve(chains, reqs, budget=sizes[-1] - 1)
    assert stats.get("checkpointed", 0) > 0
    for r, a, b in zip(reqs, base, got):
        assert not isinstance(b, Exception)
        assert a.logl == b.logl
        if r.gradient:
            assert np.array_equal(a.gradient, b.gradient)
    # below even the checkpointed form the chain's requests are rejected
    wb = chains[big]
    nb = best_band(wb.tree.children, wb.tree.n_tips)[1]
    tight = footprint(wb.tree.n_tips, wb.n_patterns, wb.n_states,
                      "f32" if wb.n_states == 4 else "tf32x3", nb) - 1
    got, stats, _ = serve(chains, reqs, budget=tight)
    for r, b in zip(reqs, got):
        if r.chain == big:
            assert isinstance(b, MemoryError)
