"""HMC over the random-effects clock (Sections 3.2 and 4.2) on the library: log pi, its gradient
and the negative Hessian diagonal in theta = log eps agree with the FP64 oracle through the chain
rule; with every pattern weight zero the posterior is the prior, the adapted mass is exactly the
prior precision and the samples have the prior's moments; a short run on data accepts and stays
finite."""
import math

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


def _target(ctx, pr, psi=0.5):
    from paper_1905_12146_gb300 import hmc
    h = ctx.upload(pr, "fp64")
    return h, hmc.ClockTarget(h, pr["parent"], pr["node_time"], pr["mu"], psi)


def test_target_matches_the_oracle(ctx, oracle_mod):
    pr = wl.config_clock_batch(seed=41, n_trees=1, n_tips=14, n_patterns=400)[0]
    h, tg = _target(ctx, pr)
    try:
        rng = np.random.default_rng(0)
        theta = tg.m + 0.3 * rng.standard_normal(tg.dim)
        logp, grad = tg.logp_grad(theta)
        nh = tg.neg_hess_diag(theta)
    finally:
        h.close()
    b = np.zeros(pr["parent"].shape[0])
    b[tg.nodes] = pr["mu"] * np.exp(theta) * tg.dt
    ref = oracle_mod.evaluate(pr, b)
    d = theta - tg.m
    lp_ref = ref.logL - 0.5 * d @ d / tg.s2 - 0.5 * tg.dim * math.log(2 * math.pi * tg.s2)
    bn, g, hh = b[tg.nodes], ref.grad[tg.nodes], ref.hess[tg.nodes]
    assert abs(logp - lp_ref) <= 1e-11 * abs(lp_ref)
    np.testing.assert_allclose(grad, bn * g - d / tg.s2, rtol=1e-9, atol=1e-9 * np.abs(bn * g).max())
    np.testing.assert_allclose(nh, -(bn * g + bn * bn * hh) + 1.0 / tg.s2, rtol=1e-8,
                               atol=1e-8 * np.abs(bn * bn * hh).max())


def test_prior_only_posterior(ctx):
    """All weights zero: logL = 0, so pi(theta) is the N(-s2/2, s2) prior in every coordinate."""
    from paper_1905_12146_gb300 import hmc
    pr = wl.config_clock_batch(seed=42, n_trees=1, n_tips=10, n_patterns=50)[0]
    pr = dict(pr, weights=np.zeros_like(pr["weights"]))
    h, tg = _target(ctx, pr, psi=0.8)
    try:
        r = hmc.hmc(tg, np.full(tg.dim, tg.m), n_iter=1500, eps=0.3, n_leapfrog=6, k=10, adapt_eps_until=200,
                    seed=5)
    finally:
        h.close()
    np.testing.assert_allclose(r["mass"], np.full(tg.dim, 1.0 / tg.s2), rtol=1e-12)
    x = r["samples"][300:]
    neff = np.array([hmc.ess(x[:, i]) for i in range(tg.dim)])
    assert neff.min() > 100
    z = (x.mean(axis=0) - tg.m) / np.sqrt(tg.s2 / neff)
    assert np.abs(z).max() < 5.0
    assert abs(np.mean(x.var(axis=0)) / tg.s2 - 1.0) < 0.1


def test_short_run_on_data(ctx):
    from paper_1905_12146_gb300 import hmc
    pr = wl.config_clock_batch(seed=43, n_trees=1, n_tips=24, n_patterns=800)[0]
    h, tg = _target(ctx, pr)
    try:
        r = hmc.hmc(tg, np.full(tg.dim, tg.m), n_iter=200, eps=0.05, n_leapfrog=8, k=10, adapt_eps_until=100,
                    seed=6)
    finally:
        h.close()
    assert np.isfinite(r["samples"]).all()
    assert 0.3 < r["accepted"][100:].mean() <= 1.0
    assert (r["mass"] > 0).all()
    assert r["gradient_evaluations"] == 1 + 200 * 8
