"""The FP64 oracle, unchanged, on several host cores (test infrastructure, like the oracle itself:
only tests and bench.py's CPU-baseline leg use it).

Site patterns are independent given the tree and the model (Section 2.1), so one evaluation of a
pattern range is a map of ``oracle.evaluate`` over contiguous slices, one spawned process per core;
the log-likelihoods of the slices add up."""
from __future__ import annotations

import multiprocessing as mp
import os

_PROBLEM = None


def _init(problem):
    global _PROBLEM
    _PROBLEM = problem


def _slice(bounds):
    from . import oracle
    lo, hi = bounds
    return oracle.evaluate(_PROBLEM, patterns=slice(lo, hi)).logL


class OraclePool:
    def __init__(self, problem, cores: int | None = None, timeout: float = 600.0):
        self.cores = cores or len(os.sched_getaffinity(0))
        self.timeout = timeout
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_init, initargs=(problem,))

    def evaluate(self, lo: int, hi: int) -> float:
        """logL of patterns [lo, hi), the slices evaluated in parallel."""
        n = hi - lo
        k = max(1, min(self.cores, n))
        cuts = [lo + (n * i) // k for i in range(k + 1)]
        return sum(self.pool.map_async(_slice, list(zip(cuts[:-1], cuts[1:]))).get(self.timeout))

    def close(self):
        self.pool.terminate()
        self.pool.join()
