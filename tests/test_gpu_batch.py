"""Batched evaluation (tl_batch_*): many four-state instances of different
taxa and pattern counts in one launch per pass. Each instance's logL and
gradient must be bit-identical to its own single-instance calls (same tile
partition, same fixed-order reductions), hence also independent of what else
is in the batch; and they must match the FP64 oracle within the stated
tolerances."""
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


# (config, n_tips, n_patterns): mixed taxa, pattern counts (ragged tails),
# HKY and GTR
SHAPES = [("hky_8x1000", 8, 1000), ("gtr_512x100k", 37, 2049), ("gtr_512x100k", 5, 33),
          ("hky_8x1000", 64, 517), ("gtr_512x100k", 3, 1), ("gtr_512x100k", 120, 3000)]


def make(cfg, n_tips, n_pat, prec, stream=None):
    from paper_2606_27607_gb300 import TreeLikelihood
    w = synth.workload(cfg, n_tips=n_tips, n_patterns=n_pat)
    tl = TreeLikelihood(n_tips, n_pat, 4, 4, prec, stream=stream)
    tl.set_tips(w.tips)
    tl.set_model(w.model, w.params, w.freqs)
    tl.set_rates(w.rates, w.cat_weights)
    tl.set_pattern_weights(w.pattern_weights)
    tl.set_tree(w.tree.children, w.tree.edge_len)
    return w, tl


def batch_eval(batch, tls, grad):
    """logL (and gradients) of every instance through the batched calls."""
    import torch
    for tl in tls:
        tl.update_matrices(grad)
    batch.update_partials([t.inst for t in tls], [t._post for t in tls])
    out = torch.zeros(len(tls), dtype=torch.float64, device="cuda")
    batch.root_loglik_dev([t.inst for t in tls], [t.nn - 1 for t in tls], [0] * len(tls),
                          out.data_ptr())
    gs = []
    if grad:
        gs = [torch.full((t.nn,), 7.0, dtype=torch.float64, device="cuda") for t in tls]
        batch.pre_order_gradient_dev([t.inst for t in tls], [t._pre for t in tls],
                                     [0] * len(tls), [g.data_ptr() for g in gs],
                                     [t.nn for t in tls])
    torch.cuda.synchronize()
    for t in tls:
        t.inst.sync()
    return out.cpu().numpy(), [g.cpu().numpy() for g in gs]


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_equals_single_bit_exact(prec):
    from paper_2606_27607_gb300._lib import Batch
    made = [make(c, n, p, prec) for c, n, p in SHAPES]
    tls = [t for _, t in made]
    try:
        single = [t.gradient() for t in tls]
        batch = Batch()
        logl, grads = batch_eval(batch, tls, grad=True)
        for k, (l1, g1) in enumerate(single):
            assert logl[k] == l1, (k, logl[k], l1)
            assert np.array_equal(grads[k], g1), k
        # the batch launched one kernel per pass (post, root, root sums, pre,
        # gradient sums), whatever the number of instances
        assert batch.launch_count() == 5
        batch.close()
    finally:
        for t in tls:
            t.close()


def test_alone_and_in_the_mix_bit_exact():
    from paper_2606_27607_gb300._lib import Batch
    made = [make(c, n, p, "f32") for c, n, p in SHAPES]
    tls = [t for _, t in made]
    try:
        batch = Batch()
        mix_l, mix_g = batch_eval(batch, tls, grad=True)
        for k, t in enumerate(tls):
            alone_l, alone_g = batch_eval(batch, [t], grad=True)
            assert alone_l[0] == mix_l[k]
            assert np.array_equal(alone_g[0], mix_g[k])
        # a different mix and order
        sub = [tls[4], tls[0], tls[5]]
        l2, g2 = batch_eval(batch, sub, grad=True)
        for j, k in enumerate([4, 0, 5]):
            assert l2[j] == mix_l[k] and np.array_equal(g2[j], mix_g[k])
        batch.close()
    finally:
        for t in tls:
            t.close()


def test_batch_matches_oracle():
    from paper_2606_27607_gb300._lib import Batch
    made = [make(c, n, p, "f32") for c, n, p in SHAPES[:4]]
    try:
        batch = Batch()
        logl, grads = batch_eval(batch, [t for _, t in made], grad=True)
        batch.close()
        for k, (w, _) in enumerate(made):
            Q, pi, _ = om.build(w.model, w.params, w.freqs)
            want_l, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights,
                                  w.tips)
            want_g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights,
                                        w.pattern_weights, w.tips)
            assert abs(logl[k] - want_l) <= 1e-5 * abs(want_l)
            scale = np.max(np.abs(want_g))
            err = np.abs(grads[k] - want_g) / np.maximum(np.abs(want_g), 1e-3 * scale)
            assert np.max(err) <= 1e-3, k
    finally:
        for _, t in made:
            t.close()


def test_batch_orders_against_instance_streams():
    """Instances on their own streams: the batch waits for their queued work
    (matrices, uploads) and their streams wait for the batch."""
    import torch
    from paper_2606_27607_gb300._lib import Batch
    streams = [torch.cuda.Stream() for _ in range(3)]
    made = [make(c, n, p, "f32", stream=s.cuda_stream)
            for (c, n, p), s in zip(SHAPES[:3], streams)]
    tls = [t for _, t in made]
    try:
        want = [t.loglik() for t in tls]
        bs = torch.cuda.Stream()
        batch = Batch(bs.cuda_stream)
        for t in tls:
            t.update_matrices(False)
        batch.update_partials([t.inst for t in tls], [t._post for t in tls])
        with torch.cuda.stream(bs):
            out = torch.zeros(3, dtype=torch.float64, device="cuda")
        batch.root_loglik_dev([t.inst for t in tls], [t.nn - 1 for t in tls], [0, 0, 0],
                              out.data_ptr())
        bs.synchronize()
        assert list(out.cpu().numpy()) == want
        batch.close()
    finally:
        for t in tls:
            t.close()


def test_batch_errors():
    import torch
    from paper_2606_27607_gb300 import TreelikError
    from paper_2606_27607_gb300._lib import Batch
    _, a = make("hky_8x1000", 8, 100, "f32")
    _, b = make("hky_8x1000", 8, 100, "f64")
    batch = Batch()
    try:
        a.update_matrices(False)
        b.update_matrices(False)
        with pytest.raises(TreelikError, match="TL_ERR_UNSUPPORTED"):
            batch.update_partials([a.inst, b.inst], [a._post, b._post])
        with pytest.raises(TreelikError, match="TL_ERR_ARG"):
            batch.update_partials([a.inst, a.inst], [a._post, a._post])
        bad = a._post.copy()
        bad["child1"][0] = 10_000
        with pytest.raises(TreelikError, match="instance 0"):
            batch.update_partials([a.inst], [bad])
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        # nothing computed yet for the root buffer of a fresh instance
        _, fresh = make("hky_8x1000", 8, 100, "f32")
        with pytest.raises(TreelikError, match="TL_ERR_STATE"):
            batch.root_loglik_dev([fresh.inst], [fresh.nn - 1], [0], out.data_ptr())
        fresh.close()
        from paper_2606_27607_gb300 import TreeLikelihood
        codon = TreeLikelihood(4, 50, 61, 4, "tf32")
        with pytest.raises(TreelikError, match="TL_ERR_UNSUPPORTED"):
            batch.update_partials([codon.inst], [np.zeros(0, dtype=a._post.dtype)])
        codon.close()
    finally:
        batch.close()
        a.close()
        b.close()
