"""Pattern-sharded evaluation of one problem across ranks (one process per GPU).

Site patterns are independent given the tree and the model (Section 2.1: logL = sum_p w_p log L_p,
and each branch derivative is a sum over patterns, Section 2.5).  A rank therefore evaluates
the log-likelihood, gradient and Hessian diagonal of its own contiguous slice of the patterns,
and one all-reduce (sum) of 1 + 2 (2N - 1) FP64 values gives the whole problem's.  The split
depends only on P and the world size, and each rank's slice is evaluated by the same
deterministic launches, so the result is reproducible for a given world size.

``ShardedEvaluator`` takes the per-slice evaluation as a callable, so the same collective layer
serves the library on each rank's GPU (the default: an upload of the slice, ``Handle.eval``) and
any other evaluator of a sub-problem.  The collective is torch.distributed on the group the caller
initialised: NCCL across GPUs, gloo on the CPU.
"""
from __future__ import annotations

import numpy as np


def shard_bounds(n_patterns: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous slice: the first P mod world ranks take one pattern more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_patterns, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_problem(problem: dict, rank: int, world: int) -> dict:
    """The sub-problem of rank's patterns (tip codes and weights sliced; everything else shared)."""
    P = problem["weights"].shape[0]
    lo, hi = shard_bounds(P, rank, world)
    sub = dict(problem)
    sub["tip_states"] = np.ascontiguousarray(problem["tip_states"][:, lo:hi])
    sub["weights"] = np.ascontiguousarray(problem["weights"][lo:hi])
    sub["pattern_range"] = (lo, hi)
    return sub


class ShardedEvaluator:
    """logL, gradient (and Hessian diagonal) of the whole problem from this rank's slice plus one
    all-reduce.

    ``evaluate(sub, b, hess) -> dict(logL, grad[, hess])`` evaluates a sub-problem.  Without it, the
    slice is uploaded once to a library context on ``device`` (FP32 or FP64 partials per
    ``precision``) and evaluated with ``Handle.eval``.  ``dist`` is torch.distributed with an
    initialised process group, or None for a single process.  ``collective_device`` is where the
    reduced vector lives: "cpu" for gloo, a CUDA device for NCCL."""

    def __init__(self, problem: dict, dist=None, evaluate=None, precision: str = "fp32", device: int = 0,
                 collective_device="cpu"):
        self.dist = dist
        self.rank = dist.get_rank() if dist is not None else 0
        self.world = dist.get_world_size() if dist is not None else 1
        self.sub = shard_problem(problem, self.rank, self.world)
        self.n = problem["parent"].shape[0]
        self.collective_device = collective_device
        self._handle = None
        self._ctx = None
        if evaluate is None:
            from . import _native
            self._ctx = _native.Context(device)
            self._handle = self._ctx.upload(self.sub, precision)
            evaluate = lambda sub, b, hess: self._handle.eval(b, grad=True, hess=hess)   # noqa: E731
        self._evaluate = evaluate

    def __call__(self, b, hess: bool = False) -> dict:
        import torch
        r = self._evaluate(self.sub, np.asarray(b, dtype=np.float64), hess)
        parts = [np.array([r["logL"]]), np.asarray(r["grad"], dtype=np.float64)]
        if hess:
            parts.append(np.asarray(r["hess"], dtype=np.float64))
        vec = torch.from_numpy(np.concatenate(parts)).to(self.collective_device)
        if self.dist is not None and self.world > 1:
            self.dist.all_reduce(vec, op=self.dist.ReduceOp.SUM)
        v = vec.cpu().numpy()
        out = {"logL": float(v[0]), "grad": v[1:1 + self.n], "patterns": self.sub["pattern_range"]}
        if hess:
            out["hess"] = v[1 + self.n:1 + 2 * self.n]
        return out

    def close(self):
        if self._handle is not None:
            self._handle.close()
            self._handle = None
        if self._ctx is not None:
            self._ctx.close()
            self._ctx = None
