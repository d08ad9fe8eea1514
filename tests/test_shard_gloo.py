"""Sharded evaluation over pattern blocks with two gloo ranks on CPU: each
rank evaluates its block (FP64 oracle), the blocks are combined by the
library's all-reduce helper, and the result equals the whole-alignment value."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import synth
    from oracle import gradient as og, model as om, pruning as op
    from paper_2606_27607_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = synth.workload("gtr_512x100k", n_tips=12, n_patterns=301)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    lo, hi = shard.pattern_blocks(w.n_patterns, world)[rank]
    tips = w.tips[:, lo:hi]
    wt = w.pattern_weights[lo:hi]
    logl, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, wt, tips)
    g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, wt, tips)
    tot = shard.allreduce_sum(np.concatenate([[logl], g]))
    if rank == 0:
        q.put(tot)
    dist.destroy_process_group()


def test_pattern_blocks_cover_exactly():
    from paper_2606_27607_gb300 import shard
    for n, k in ((10, 3), (100_000, 8), (5, 5), (7, 1)):
        b = shard.pattern_blocks(n, k)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[i][1] == b[i + 1][0] for i in range(k - 1))
        sizes = [hi - lo for lo, hi in b]
        assert max(sizes) - min(sizes) <= 1


def test_two_rank_gloo_sum_equals_whole():
    mp = pytest.importorskip("torch.multiprocessing")
    import synth
    from oracle import gradient as og, model as om, pruning as op
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    tot = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = synth.workload("gtr_512x100k", n_tips=12, n_patterns=301)
    Q, pi, _ = om.build(w.model, w.params, w.freqs)
    logl, _ = op.loglik(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    g = og.branch_gradient(w.tree, Q, pi, w.rates, w.cat_weights, w.pattern_weights, w.tips)
    assert abs(tot[0] - logl) <= 1e-12 * abs(logl)
    assert np.allclose(tot[1:], g, rtol=1e-11, atol=1e-11)
