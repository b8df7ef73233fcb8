"""Pattern-sharded evaluation (one all-reduce of logL and the per-branch sums) with two gloo ranks on
the CPU, the FP64 oracle evaluating each rank's slice: the reduced logL, gradient and Hessian
diagonal equal the whole problem's, and the slices partition the patterns."""
import os
import socket
import sys

import numpy as np
import pytest

from paper_1905_12146_gb300 import sharded
from paper_1905_12146_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_bounds_partition_the_patterns():
    for P in (0, 1, 7, 500, 10001):
        for world in (1, 2, 3, 8):
            spans = [sharded.shard_bounds(P, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == P
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.shard_bounds(10, 2, 2)


def _oracle_eval(sub, b, hess):
    sys.path.insert(0, ROOT)
    from oracle import oracle
    r = oracle.evaluate(sub, b)
    return {"logL": r.logL, "grad": r.grad, "hess": r.hess}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pr = wl.config_small()
        ev = sharded.ShardedEvaluator(pr, dist=dist, evaluate=_oracle_eval)
        out = ev(pr["b"], hess=True)
        q.put((rank, out["logL"], out["grad"], out["hess"], out["patterns"]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_equal_the_whole_problem():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    from oracle import oracle
    oracle.build()
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    pr = wl.config_small()
    ref = oracle.evaluate(pr, pr["b"])
    P = pr["weights"].shape[0]
    assert got[0][4] == (0, P // 2 + P % 2) and got[1][4][1] == P
    for _, logL, grad, hess, _ in got:   # every rank holds the reduced result
        assert abs(logL - ref.logL) <= 1e-12 * abs(ref.logL)
        np.testing.assert_allclose(grad, ref.grad, rtol=1e-10, atol=1e-10 * np.abs(ref.grad).max())
        np.testing.assert_allclose(hess, ref.hess, rtol=1e-9, atol=1e-9 * np.abs(ref.hess).max())


def test_slices_keep_the_tip_vector_table():
    """A slice keeps the problem's tip-vector table (partially observed tips), so the slices'
    oracle results sum to the whole problem's."""
    sys.path.insert(0, ROOT)
    from oracle import oracle
    pr = wl.random_problem(12, 90, n_states=4, n_cat=2, seed=81, b_mean=0.1, ambiguous=0.05)
    table = wl.iupac_nucleotide_partials(error=0.02)
    pr = dict(pr, tip_partials=table,
              tip_states=wl.make_partially_observed(pr["tip_states"], 0.2, table, np.random.default_rng(81)))
    ref = oracle.evaluate(pr)
    parts = [oracle.evaluate(sharded.shard_problem(pr, r, 3)) for r in range(3)]
    assert abs(sum(p.logL for p in parts) - ref.logL) <= 1e-12 * abs(ref.logL)
    np.testing.assert_allclose(sum(p.grad for p in parts), ref.grad, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(sum(p.hess for p in parts), ref.hess, rtol=1e-9, atol=1e-10)
