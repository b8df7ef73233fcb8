"""Evaluation under a device-memory budget smaller than the problem's arrays.

A problem whose partials do not fit the context's budget is evaluated in contiguous pattern chunks
(sites are i.i.d., Section 2.1, so logL, gradient and Hessian diagonal are sums over pattern
slices) that share one region for their partials; the backward half of an autograd pair recomputes
each chunk's post-order partials before its pre-order pass.  Results must match the FP64 oracle
within the paths' parity bounds and the unconstrained evaluation to FP32 rounding.
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


def _maxrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _full_bytes(native, pr, precision="fp32"):
    ctx = native.Context(0)
    h = ctx.upload(pr, precision)
    try:
        info = h.info()
        ref = h.eval(pr["b"], grad=True, hess=True, site=True)
    finally:
        h.close()
        ctx.close()
    return info.device_bytes, ref


@pytest.mark.parametrize("m,n_tips,n_pat,n_cat,precision,frac", [(4, 120, 3000, 4, "fp32", 0.45),
                                                                  (4, 60, 1500, 2, "fp64", 0.45),
                                                                  (61, 30, 2000, 2, "fp32", 0.6)])
def test_budget_below_the_partials_evaluates_in_chunks(native, oracle_mod, m, n_tips, n_pat, n_cat, precision, frac):
    pr = wl.random_problem(n_tips, n_pat, n_states=m, n_cat=n_cat, seed=400 + m, b_mean=0.05 if m == 4 else 0.1,
                           ambiguous=0.03)
    whole, plain = _full_bytes(native, pr, precision)
    ctx = native.Context(0, hbm_budget_bytes=int(frac * whole))
    try:
        h = ctx.upload(pr, precision)   # does not fit whole: pattern chunks
        try:
            info = h.info()
            assert info.device_bytes <= frac * whole and info.n_patterns == n_pat
            got = h.eval(pr["b"], grad=True, hess=True, site=True)
        finally:
            h.close()
    finally:
        ctx.close()
    ref = oracle_mod.evaluate(pr)
    assert got["status"] == 0
    n_int = n_tips - 1
    if precision == "fp64":
        lb, gb, hb = 1e-12 * abs(ref.logL), 1e-11, 1e-10
    elif m == 4:
        lb = max(1e-9 * abs(ref.logL), 6 * 2.0 ** -24 * np.sqrt(n_int * np.sum(pr["weights"] ** 2)))
        gb, hb = 1e-5, 1e-4
    else:
        lb = 16.0 * np.sqrt(n_int) * (np.sqrt(m) + 1.0) * 2.0 ** -24 * np.sum(pr["weights"])
        gb, hb = 1e-5, 2e-5
    print(f"m={m} {precision}: budget {frac * whole / 1e6:.1f} MB of {whole / 1e6:.1f}, held {info.device_bytes / 1e6:.1f}; "
          f"logL abs {abs(got['logL'] - ref.logL):.2e}  grad {_maxrel(got['grad'], ref.grad):.2e}  "
          f"hess {_maxrel(got['hess'], ref.hess):.2e}")
    assert abs(got["logL"] - ref.logL) <= lb
    assert _maxrel(got["grad"], ref.grad) <= gb
    assert _maxrel(got["hess"], ref.hess) <= hb
    # against the evaluation of the whole problem: the same arithmetic per pattern
    np.testing.assert_allclose(got["site_logL"], plain["site_logL"], rtol=0, atol=1e-12 if precision == "fp64" else
                               16.0 * np.sqrt(n_int) * (np.sqrt(m) + 1.0) * 2.0 ** -24)
    assert _maxrel(got["grad"], plain["grad"]) <= gb


def test_chunked_forward_backward_recomputes_the_partials(native):
    """The autograd halves on a chunked problem: the backward recomputes each chunk's partials for
    the branch lengths of the forward (even if the caller's array changed since) and gives the
    gradient of one evaluation bit for bit; batched calls take chunked problems too."""
    import torch
    dev = torch.device("cuda")
    pr = wl.random_problem(100, 2500, n_states=4, n_cat=4, seed=410, b_mean=0.05, ambiguous=0.03)
    whole, _ = _full_bytes(native, pr)
    ctx = native.Context(0, hbm_budget_bytes=int(0.4 * whole) + (8 << 20))
    h2 = ctx.upload(wl.random_problem(20, 300, n_states=4, n_cat=4, seed=411))   # first: the chunks take what is left
    h = ctx.upload(pr)
    assert h.info().device_bytes < whole
    try:
        b = torch.tensor(pr["b"], device=dev)
        l0 = torch.zeros(1, dtype=torch.float64, device=dev)
        g0 = torch.zeros_like(b)
        h.eval_async(b, l0, g0)
        l1 = torch.zeros(1, dtype=torch.float64, device=dev)
        g1 = torch.zeros_like(b)
        h.forward_async(b, l1)
        b2 = b.clone()
        b.mul_(3.0)                              # the forward's lengths are what the backward uses
        h.backward_async(None, g1)
        torch.cuda.synchronize()
        assert h.status() == 0
        assert l1.item() == l0.item()
        assert torch.equal(g1, g0)
        # a batch with a chunked and a whole problem
        bs = [b2, torch.tensor(wl.random_problem(20, 300, n_states=4, n_cat=4, seed=411)["b"], device=dev)]
        logL = torch.zeros(2, dtype=torch.float64, device=dev)
        gs = [torch.zeros_like(bs[0]), torch.zeros_like(bs[1])]
        native.eval_batch_async([h, h2], bs, logL, d_grad=gs)
        torch.cuda.synchronize()
        assert h.status() == 0 and h2.status() == 0
        assert logL[0].item() == l0.item() and torch.equal(gs[0], g0)
    finally:
        h.close()
        h2.close()
        ctx.close()


def test_budget_too_small_even_for_chunks(native):
    pr = wl.random_problem(200, 2000, n_states=4, n_cat=4, seed=420)
    ctx = native.Context(0, hbm_budget_bytes=1 << 20)
    try:
        with pytest.raises(native.PhyloGradError) as e:
            ctx.upload(pr)
        assert e.value.status == native.PG_ERR_OOM
        assert "chunks" in native.load().pg_last_error().decode()
    finally:
        ctx.close()
