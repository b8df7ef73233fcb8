"""torch.autograd.Functions over the CUDA library (argument marshalling only).

``TreeLogLikelihood``: the forward is the pruning pass (post-order partials, Section 2.3, and the
root mixture, Section 2.5) and the backward is the pre-order pass with the branch gradient
(Sections 2.4-2.5), scaled on the device by the upstream gradient.  The post-order partials of
the forward stay resident in each problem's handle; if another forward ran on a handle before the
backward, the backward first recomputes that handle's forward for the saved branch lengths.

``ClockBranchLengths``: the random-effects clock b_i = mu * eps_i * (t_i - t_parent(i)) of
Sections 2.1 and 5.1, with its chain rule to eps, mu and the node times in the backward.

Both run every arithmetic step in libphylograd.so kernels on the current CUDA stream; there is no
CPU path.  Inputs are float64 CUDA tensors of shape [k, 2N-1] (k problems with the same node
count; row i belongs to handles[i]) and [k] for mu.
"""
from __future__ import annotations

import torch

from . import _native


def _bump(h):
    h._fwd_gen = getattr(h, "_fwd_gen", 0) + 1
    return h._fwd_gen


def _forward(handles, b, logL, stream):
    if len(handles) == 1:
        handles[0].forward_async(b[0], logL, stream=stream)
    else:
        _native.forward_batch_async(handles, [b[i] for i in range(len(handles))], logL, stream=stream)


def _check_rows(x, handles, name):
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if x.dim() != 2 or x.shape[0] != len(handles):
        raise ValueError(f"{name} must have shape [k, 2N-1] with k = {len(handles)}")
    for h in handles:
        if h.n_nodes != x.shape[1]:
            raise ValueError(f"{name}: every problem of a call must have {x.shape[1]} nodes")


class TreeLogLikelihood(torch.autograd.Function):
    """logL[i] of problem i for branch lengths b[i]; backward gives dlogL/db times grad_output."""

    @staticmethod
    def forward(ctx, b, handles):
        handles = tuple(handles)
        _check_rows(b, handles, "b")
        b = b.contiguous()
        stream = torch.cuda.current_stream(b.device)
        logL = torch.empty(len(handles), dtype=torch.float64, device=b.device)
        _forward(handles, b, logL, stream)
        ctx.handles = handles
        ctx.gens = tuple(_bump(h) for h in handles)
        ctx.save_for_backward(b)
        return logL

    @staticmethod
    def backward(ctx, g):
        (b,) = ctx.saved_tensors
        handles = ctx.handles
        stream = torch.cuda.current_stream(b.device)
        stale = [i for i, h in enumerate(handles) if h._fwd_gen != ctx.gens[i]]
        if stale:   # another forward replaced the resident partials: recompute them
            hs = tuple(handles[i] for i in stale)
            scratch = torch.empty(len(hs), dtype=torch.float64, device=b.device)
            _forward(hs, b[stale].contiguous(), scratch, stream)
            for h in hs:
                _bump(h)
        g = g.to(torch.float64).contiguous()
        grad = torch.empty_like(b)
        if len(handles) == 1:
            handles[0].backward_async(g, grad[0], stream=stream)
        else:
            _native.backward_batch_async(handles, g, [grad[i] for i in range(len(handles))], stream=stream)
        return grad, None


class ClockBranchLengths(torch.autograd.Function):
    """b[i, j] = mu[i] * eps[i, j] * (t[i, j] - t[i, parent(j)]), 0 at the root."""

    @staticmethod
    def forward(ctx, eps, mu, t, handles):
        handles = tuple(handles)
        _check_rows(eps, handles, "eps")
        _check_rows(t, handles, "t")
        if mu.shape != (len(handles),) or mu.dtype != torch.float64:
            raise ValueError("mu must be a float64 tensor of shape [k]")
        eps, mu, t = eps.contiguous(), mu.contiguous(), t.contiguous()
        k = len(handles)
        b = torch.empty_like(eps)
        _native.clock_lengths_async(handles, [eps[i] for i in range(k)], mu, [t[i] for i in range(k)],
                                    [b[i] for i in range(k)], stream=torch.cuda.current_stream(eps.device))
        ctx.handles = handles
        ctx.save_for_backward(eps, mu, t)
        return b

    @staticmethod
    def backward(ctx, gb):
        eps, mu, t = ctx.saved_tensors
        handles = ctx.handles
        k = len(handles)
        gb = gb.to(torch.float64).contiguous()
        need_eps, need_mu, need_t = ctx.needs_input_grad[:3]
        g_eps = torch.empty_like(eps) if need_eps else None
        g_mu = torch.empty_like(mu) if need_mu else None
        g_t = torch.empty_like(t) if need_t else None
        rows = lambda x: None if x is None else [x[i] for i in range(k)]
        _native.clock_grad_async(handles, rows(eps), mu, rows(t), rows(gb), d_grad_eps=rows(g_eps),
                                 d_grad_mu=g_mu, d_grad_t=rows(g_t),
                                 stream=torch.cuda.current_stream(eps.device))
        return g_eps, g_mu, g_t, None


def tree_loglik(b, handles):
    """logL [k] of k problems (TreeLogLikelihood.apply)."""
    return TreeLogLikelihood.apply(b, tuple(handles))


def clock_branch_lengths(eps, mu, t, handles):
    """Branch lengths [k, 2N-1] of the random-effects clock (ClockBranchLengths.apply)."""
    return ClockBranchLengths.apply(eps, mu, t, tuple(handles))


def check_status(handles):
    """Wait for each handle's last evaluation and raise on a device-side error status."""
    for h in handles:
        st = h.status()
        if st != _native.PG_OK:
            _native.check(st)
