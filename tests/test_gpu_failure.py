"""Failure detection without a GPU fault: the library's bounded device-side wait, run on a barrier
that nothing arrives at, gives up after its limit and reports PG_ERR_TIMEOUT through the status
path every kernel uses; the context stays usable (an evaluation right after it is correct)."""
import time

import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_12146_gb300 import _native, build
    build.build()
    c = _native.Context(0)
    yield c
    c.close()


def test_bounded_wait_times_out_and_context_survives(ctx, oracle_mod):
    from paper_1905_12146_gb300 import _native
    t0 = time.perf_counter()
    st = ctx.selftest_timeout(2_000_000)   # ~1 ms of SM clocks
    assert st == _native.PG_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert ctx.selftest_timeout(20_000_000) == _native.PG_ERR_TIMEOUT
    pr = wl.config_small()
    h = ctx.upload(pr, "fp64")
    try:
        r = h.eval(pr["b"], grad=True)
    finally:
        h.close()
    ref = oracle_mod.evaluate(pr, pr["b"])
    assert r["status"] == 0
    assert abs(r["logL"] - ref.logL) <= 1e-12 * abs(ref.logL)
    np.testing.assert_allclose(r["grad"], ref.grad, rtol=1e-10, atol=1e-10 * np.abs(ref.grad).max())


def test_selftest_rejects_bad_limits(ctx):
    from paper_1905_12146_gb300 import _native
    assert ctx.selftest_timeout(10) == _native.PG_ERR_INVALID
    assert ctx.selftest_timeout(1 << 40) == _native.PG_ERR_INVALID
