"""torch.autograd.Function over the library: forward = post-order pass and
root log-likelihood; backward = one pre-order pass and one adjoint pass,
which give dlogL/dt for every branch and dlogL/dQ, hence every
substitution parameter (Sec. "Algorithmic advances": linear-time gradients;
Sec. "Discussion": exact substitution gradients through the adjoint of the
matrix exponential). All arithmetic runs in the library's kernels; this
module moves tensors across the boundary."""
from __future__ import annotations

import numpy as np
import torch


class LogLikelihood(torch.autograd.Function):
    """logL(t, theta) for a TreeLikelihood whose tips, frequencies, rates and
    topology are set. ``edge_len`` holds one length per non-root node;
    ``params`` are the model parameters (kappa | six GTR exchangeabilities |
    kappa, omega | kappa, omega and 263 random effects | the S x S
    exchangeabilities of a general reversible model). Returns a 0-d float64
    tensor."""

    @staticmethod
    def forward(ctx, edge_len: torch.Tensor, params: torch.Tensor, tl, kind: str, freqs):
        if params.requires_grad and kind not in ("hky", "gtr", "gy94", "gy94re", "rev"):
            raise ValueError(f"model {kind!r} has no parameter derivatives; take dlogL/dQ from "
                             "TreeLikelihood.adjoint() instead")
        t = edge_len.detach().cpu().double().numpy()
        th = params.detach().cpu().double().numpy()
        LogLikelihood._evaluate(tl, kind, th, freqs, t)
        ctx.tl = tl
        ctx.dev = edge_len.device
        ctx.saved = (kind, th, freqs, t)
        ctx.generation = tl.generation
        return torch.tensor(tl.last_logl, dtype=torch.float64)

    @staticmethod
    def _evaluate(tl, kind, th, freqs, t):
        tl.set_model(kind, th, freqs)
        full = np.zeros(tl.nn)
        full[: tl.nn - 1] = t
        tl.set_tree(tl.children, full)
        tl.last_logl = tl.loglik()

    @staticmethod
    def backward(ctx, grad_out):
        tl = ctx.tl
        # The adjoint reads the post-order partials and matrices on the
        # device. They are this forward's unless another evaluation on the
        # same instance ran since (two forwards before one backward, a
        # finite-difference probe in between): then this forward's state is
        # rebuilt from its saved inputs first.
        if tl.generation != ctx.generation:
            LogLikelihood._evaluate(tl, *ctx.saved)
        g, _, gth = tl.adjoint()
        s = float(grad_out)
        gt = torch.from_numpy(s * g[: tl.nn - 1]).to(ctx.dev)
        gp = torch.from_numpy(s * gth).to(ctx.dev)
        return gt, gp, None, None, None
