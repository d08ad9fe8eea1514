"""The op lists of subtree checkpointing, checked on the host by simulating
which node each buffer holds: every op reads its children's post-order
partials and its parent's pre-order partial from buffers that hold them at
that moment (written earlier in the list or by an earlier call), each list
writes a buffer at most once, pre-order partials never share buffers with
post-order ones, every edge's derivative comes from exactly one band, and
the buffer count is below the whole-tree count on large trees."""
import numpy as np
import pytest

import synth
from paper_2606_27607_gb300.checkpoint import CheckpointedLikelihood, best_band


def run_post(ops, holds, parent):
    dests = [int(d) for d in ops["dest"]]
    assert len(set(dests)) == len(dests)
    for o in ops:
        for c, m in ((int(o["child1"]), int(o["mat1"])), (int(o["child2"]), int(o["mat2"]))):
            assert holds.get(c) == m, (c, m, holds.get(c))
        holds[int(o["dest"])] = int(parent[int(o["mat1"])])


@pytest.mark.parametrize("name,n_tips", [("gtr_512x100k", 512), ("gtr_1024x50k", 300),
                                         ("gy94_128x20k", 128), ("gy94_64x5k", 9)])
@pytest.mark.parametrize("band", [1, 2, 3, 4, 6])
def test_checkpoint_op_lists(name, n_tips, band):
    w = synth.workload(name, n_tips=n_tips, n_patterns=4)
    N = w.tree.n_tips
    nn = 2 * N - 1
    parent = np.asarray(w.tree.parent)
    ck = CheckpointedLikelihood(N, 4, w.tree.children, band=band, create=False)
    holds = {t: t for t in range(N)}           # post-order buffer -> node
    for b in range(len(ck.bands) - 1, -1, -1):  # forward, bottom-up
        run_post(ck.post_ops[b], holds, parent)
    assert holds.get(ck.ck_buf[nn - 1]) == nn - 1
    qholds, edges = {}, []
    q_range = set(range(ck.q_base, ck.q_base + ck.q_size))
    for b in range(len(ck.bands)):              # backward, top-down
        if b > 0:
            run_post(ck.re_ops[b], holds, parent)
        pre = ck.pre_ops[b]
        outs = [int(x) for o in pre for x in o["pre"] if x >= 0]
        assert len(set(outs)) == len(outs) and set(outs) <= q_range
        for o in pre:                           # listed parent first
            node = int(parent[int(o["mat"][0])])
            if node == nn - 1:
                assert o["parent_pre"] == -1
            else:
                assert qholds.get(int(o["parent_pre"])) == node
            for c in range(2):
                assert holds.get(int(o["child"][c])) == int(o["mat"][c])
                assert o["dmat"][c] == nn + o["mat"][c]
                edges.append(int(o["edge"][c]))
                if o["pre"][c] >= 0:
                    qholds[int(o["pre"][c])] = int(o["mat"][c])
    assert sorted(edges) == list(range(nn - 1))
    if N >= 128 and band in (2, 3, 4):
        assert ck.n_buffers < 0.75 * 2 * (N - 1)


def test_best_band_saves_buffers_on_the_benchmark_trees():
    for name in ("gtr_512x100k", "gtr_1024x50k", "gy94_128x20k"):
        w = synth.workload(name, n_patterns=4)
        band, nb = best_band(w.tree.children, w.tree.n_tips)
        assert nb <= 0.6 * 2 * (w.tree.n_tips - 1), (name, band, nb)


def test_checkpointed_footprint_admits_what_the_whole_tree_cannot():
    """The server's footprint with checkpoint buffers is the smaller one it
    compares against its budget."""
    pytest.importorskip("torch")
    from paper_2606_27607_gb300.serve import footprint
    w = synth.workload("gy94_128x20k", n_patterns=4)
    band, nb = best_band(w.tree.children, w.tree.n_tips)
    whole = footprint(w.tree.n_tips, 20000, 61, "tf32x2")
    ck = footprint(w.tree.n_tips, 20000, 61, "tf32x2", nb)
    assert ck < 0.6 * whole
    assert footprint(w.tree.n_tips, 20000, 61, "tf32x2", 2 * (w.tree.n_tips - 1)) == whole
