"""Maximum-likelihood branch-specific rates by L-BFGS (Section 3) on the CUDA library.

Branch lengths follow Section 2.1, b_i = r_i (t_i - t_parent(i)), with fixed node times and one
free rate per branch, optimised as theta_i = log r_i (positive parameters are log-transformed,
Section 3).  The objective is -logL.  Two gradients are compared, as in the paper's Table 1:

* ``analytic``: the backward pass of ``autograd.TreeLogLikelihood`` (pre-order pass and branch
  gradient, Sections 2.4-2.5) through ``autograd.ClockBranchLengths`` (b = mu eps dt with mu = 1,
  eps = r), O(N) per gradient;
* ``numeric``: central differences of logL in every theta_i, two forward (post-order) passes per
  rate, O(N^2) per gradient.

Every likelihood and gradient evaluation runs in the library's kernels; the L-BFGS iteration
(two-loop recursion, strong-Wolfe line search) is torch.optim.LBFGS around them.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import autograd


def rate_mle(handle, node_times, log_rates0, method: str = "analytic", max_iter: int = 200,
             tolerance_grad: float = 1e-7, tolerance_change: float = 1e-12, h: float = 1e-6,
             history_size: int = 10):
    """Maximise logL over theta = log r for the problem in ``handle`` (one tree).

    ``node_times`` [2N-1] in forward time; ``log_rates0`` [2N-1] the start (the root's entry is
    not a parameter).  Returns a dict with theta, logL, L-BFGS iterations, objective evaluations,
    forward passes and wall seconds.
    """
    if method not in ("analytic", "numeric"):
        raise ValueError("method must be 'analytic' or 'numeric'")
    dev = torch.device("cuda", handle.ctx.device)
    hs = [handle]
    n, root = handle.n_nodes, handle.root
    t = torch.tensor(np.asarray(node_times, dtype=np.float64), device=dev)[None]
    mu = torch.ones(1, dtype=torch.float64, device=dev)
    theta = torch.tensor(np.asarray(log_rates0, dtype=np.float64), device=dev)[None].requires_grad_(True)
    stats = {"objective": 0, "forward_passes": 0}

    def logl_of(th):
        stats["forward_passes"] += 1
        return autograd.tree_loglik(autograd.clock_branch_lengths(torch.exp(th), mu, t, hs), hs)

    def closure():
        opt.zero_grad()
        stats["objective"] += 1
        if method == "analytic":
            loss = -logl_of(theta).sum()
            loss.backward()
            theta.grad[0, root] = 0.0
            return loss
        with torch.no_grad():
            loss = -logl_of(theta).sum()
            g = torch.zeros_like(theta)
            for i in range(n):
                if i == root:
                    continue
                tp, tm = theta.clone(), theta.clone()
                tp[0, i] += h
                tm[0, i] -= h
                g[0, i] = -(logl_of(tp).sum() - logl_of(tm).sum()) / (2 * h)
            theta.grad = g
        return loss

    opt = torch.optim.LBFGS([theta], lr=1.0, max_iter=max_iter, tolerance_grad=tolerance_grad,
                            tolerance_change=tolerance_change, history_size=history_size,
                            line_search_fn="strong_wolfe")
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    opt.step(closure)
    torch.cuda.synchronize(dev)
    seconds = time.perf_counter() - t0
    autograd.check_status(hs)
    state = opt.state[theta]
    with torch.no_grad():
        final = logl_of(theta).item()
    return {"theta": theta.detach()[0].cpu().numpy(), "logL": final, "iterations": int(state.get("n_iter", 0)),
            "objective_evaluations": stats["objective"], "forward_passes": stats["forward_passes"],
            "seconds": seconds, "method": method}
