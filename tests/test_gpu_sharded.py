"""Pattern slices on the library: the slices' logL, gradient and Hessian diagonal add up to the
whole problem's (FP64 partials: to rounding; FP32: within the FP32 bound), and a single-rank
ShardedEvaluator is the plain evaluation bit for bit."""
import numpy as np
import pytest

from paper_1905_12146_gb300 import sharded
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


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_slices_add_up(ctx, precision, rtol):
    pr = wl.config_small()
    whole = ctx.upload(pr, precision)
    try:
        ref = whole.eval(pr["b"], grad=True, hess=True)
    finally:
        whole.close()
    tot = {"logL": 0.0, "grad": 0.0, "hess": 0.0}
    for r in range(3):
        h = ctx.upload(sharded.shard_problem(pr, r, 3), precision)
        try:
            out = h.eval(pr["b"], grad=True, hess=True)
        finally:
            h.close()
        for k in tot:
            tot[k] = tot[k] + out[k]
    assert abs(tot["logL"] - ref["logL"]) <= rtol * abs(ref["logL"])
    np.testing.assert_allclose(tot["grad"], ref["grad"], rtol=rtol, atol=rtol * np.abs(ref["grad"]).max())
    np.testing.assert_allclose(tot["hess"], ref["hess"], rtol=10 * rtol, atol=10 * rtol * np.abs(ref["hess"]).max())


def test_single_rank_is_the_plain_evaluation(ctx):
    pr = wl.config_small()
    ev = sharded.ShardedEvaluator(pr, dist=None, precision="fp32")
    try:
        out = ev(pr["b"], hess=True)
    finally:
        ev.close()
    h = ctx.upload(pr, "fp32")
    try:
        ref = h.eval(pr["b"], grad=True, hess=True)
    finally:
        h.close()
    assert out["logL"] == ref["logL"]
    np.testing.assert_array_equal(out["grad"], ref["grad"])
    np.testing.assert_array_equal(out["hess"], ref["hess"])
