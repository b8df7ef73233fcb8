"""The allocation-free entry point (pg_eval_noalloc) against the regular one (pg_eval).

pg_eval_noalloc is for callers that cannot allocate when they evaluate: it keeps every
intermediate array in one fixed device array per GPU and plans on fixed host buffers.  This file
is collected last so that a run stopping at its first failure has run every other test already.
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_12146_gb300 import _native, build
    build.build()
    return _native


def _regular(native, pr, precision):
    ctx = native.Context(0)
    h = ctx.upload(pr, precision)
    out = h.eval(pr["b"], grad=True, hess=True, site=True)
    h.close()
    ctx.close()
    return out


@pytest.mark.parametrize("precision,logl_rtol,grad_rtol", [("fp64", 1e-12, 1e-11), ("fp32", 1e-9, 1e-5)])
def test_noalloc_matches_pg_eval_on_two_calls_in_a_row(native, oracle_mod, precision, logl_rtol, grad_rtol):
    """Two different problems in a row through the shared scratch array: each result matches the
    regular entry point and the FP64 oracle within the parity tolerances (the second call must not
    see the first's leftovers)."""
    problems = [wl.random_problem(40, 777, n_states=4, n_cat=4, seed=301, b_mean=0.05, ambiguous=0.03,
                                  weights="int"),
                wl.config_small(seed=2)]
    for pr in problems:
        ref = _regular(native, pr, precision)
        orc = oracle_mod.evaluate(pr, pr["b"])
        got = native.eval_noalloc(pr, pr["b"], precision, grad=True, hess=True, site=True)
        assert got["status"] == 0
        # FP32 rounding noise of small problems: one rounding per internal node and site
        lbound = max(logl_rtol * abs(orc.logL),
                     6 * 2.0 ** -24 * np.sqrt((pr["n_tips"] - 1) * np.sum(pr["weights"] ** 2)))
        for other in (ref, {"logL": orc.logL, "grad": orc.grad, "hess": orc.hess, "site_logL": orc.site_logL}):
            assert abs(got["logL"] - other["logL"]) <= lbound
            assert np.abs(got["grad"] - other["grad"]).max() <= grad_rtol * np.abs(other["grad"]).max()
            assert np.abs(got["hess"] - other["hess"]).max() <= 10 * grad_rtol * np.abs(other["hess"]).max()
            np.testing.assert_allclose(got["site_logL"], other["site_logL"], rtol=0,
                                       atol=1e-10 if precision == "fp64" else 6 * (pr["n_tips"] - 1) * 2.0 ** -24)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_outputs_beyond_the_static_image(native, oracle_mod, precision):
    """150,000 site likelihoods (1.2 MB, over the 1 MiB static host image of the outputs) come back
    array by array; they and logL match the regular entry point."""
    pr = wl.random_problem(5, 150000, n_states=4, n_cat=1, seed=305, b_mean=0.1, ambiguous=0.02)
    ref = _regular(native, pr, precision)
    got = native.eval_noalloc(pr, pr["b"], precision, grad=True, hess=True, site=True)
    assert got["status"] == 0
    tol = 1e-12 if precision == "fp64" else 6 * 4 * 2.0 ** -24
    np.testing.assert_allclose(got["site_logL"], ref["site_logL"], rtol=0, atol=tol)
    assert abs(got["logL"] - ref["logL"]) <= (1e-12 if precision == "fp64" else 1e-7) * abs(ref["logL"])
    assert np.abs(got["grad"] - ref["grad"]).max() <= 1e-5 * np.abs(ref["grad"]).max()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_without_patterns(native, precision):
    """No site patterns: logL, gradient and Hessian diagonal are exactly zero, as from pg_eval."""
    pr = wl.config_small(seed=3)
    pr = dict(pr, tip_states=pr["tip_states"][:, :0], weights=pr["weights"][:0])
    got = native.eval_noalloc(pr, pr["b"], precision, grad=True, hess=True, site=True)
    assert got["status"] == 0
    assert got["logL"] == 0.0
    assert not got["grad"].any() and not got["hess"].any()
    ref = _regular(native, pr, precision)
    assert ref["logL"] == 0.0 and not ref["grad"].any()


def test_noalloc_rejects_problems_beyond_its_scratch(native):
    """A problem larger than the fixed scratch array is refused with a message (recorded in a
    static buffer, without allocating) that pg_last_error returns on the calling thread."""
    pr = wl.random_problem(300, 20000, n_states=4, n_cat=4, seed=302, b_mean=0.05)
    with pytest.raises(native.PhyloGradError) as e:
        native.eval_noalloc(pr, pr["b"], "fp32")
    assert e.value.status == native.PG_ERR_UNSUPPORTED
    assert "scratch" in native.load().pg_last_error().decode()
