"""tl_root_loglik_static: the root log-likelihood for callers that cannot
allocate device memory (inside another component's stream capture, plug-ins
whose host owns the allocator, allocation-free real-time loops). Its scratch
is a fixed array built into the library. Checked against tl_root_loglik of
an instance on the same data, twice in a row (the shared scratch keeps the
previous call's contents). Collected last so a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_static_root_loglik_matches_instance_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import TreeLikelihood, build, _lib
    build.build()
    stream = torch.cuda.current_stream()
    for n_tips, n_pat in ((30, 1000 + 13), (12, 70)):
        w = synth.workload("gtr_512x100k", n_tips=n_tips, n_patterns=n_pat)
        tl = TreeLikelihood(n_tips, n_pat, 4, 4, "f32", stream=stream.cuda_stream)
        tl.set_tips(w.tips)
        tl.set_model(w.model, w.params, w.freqs)
        tl.set_rates(w.rates, w.cat_weights)
        wts = np.random.default_rng(1).integers(1, 4, size=n_pat).astype(float)
        tl.set_pattern_weights(wts)
        tl.set_tree(w.tree.children, w.tree.edge_len)
        want = tl.loglik()
        root = 2 * n_tips - 2
        part, exps = tl.inst.get_partials(root)           # FP32 values, exactly
        Q, pi, _ = tl.inst.get_model(0)
        tl.close()
        stride = (n_pat + 31) // 32 * 32
        buf = np.zeros((4, stride, 4), dtype=np.float32)
        buf[:, :n_pat, :] = part.astype(np.float32)
        d_root = torch.from_numpy(buf).cuda()
        d_exps = torch.from_numpy(exps.astype(np.int32)).cuda()
        d_pi = torch.from_numpy(pi).cuda()
        d_cw = torch.from_numpy(np.asarray(w.cat_weights, float)).cuda()
        d_pw = torch.from_numpy(wts).cuda()
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        for k in range(2):
            _lib.root_loglik_static(d_root.data_ptr(), d_exps.data_ptr(), d_pi.data_ptr(),
                                    d_cw.data_ptr(), d_pw.data_ptr(), n_pat, stride, 4,
                                    out.data_ptr() + 8 * k, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-12 * abs(want)), (got, want)


def test_static_root_loglik_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_27607_gb300 import _lib
    x = torch.zeros(16, dtype=torch.float32, device="cuda")
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.TreelikError, match="TL_ERR_UNSUPPORTED"):
        _lib.root_loglik_static(x.data_ptr(), None, d.data_ptr(), d.data_ptr(), d.data_ptr(),
                                2_097_153, 2_097_184, 4, d.data_ptr())
