"""The HMC sampler of Section 3.2 on targets with known answers (CPU only): the effective sample
size estimator on AR(1) chains, leapfrog reversibility and second-order energy error, the moments
of an anisotropic Gaussian with the adaptive diagonal mass matrix, and the mass update rule of
Section 3.2.1 (running mean of the Hessian diagonal every k iterations, clamped)."""
import numpy as np
import pytest

from paper_1905_12146_gb300 import hmc


class Gaussian:
    """log N(theta; mean, diag(sd^2)); -d^2 log pi / d theta^2 = 1 / sd^2."""

    def __init__(self, mean, sd):
        self.mean, self.sd = np.asarray(mean, float), np.asarray(sd, float)

    def logp_grad(self, th):
        z = (th - self.mean) / self.sd
        return -0.5 * float(z @ z), -z / self.sd

    def neg_hess_diag(self, th):
        return 1.0 / self.sd ** 2


def ar1(n, rho, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    return x


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_of_ar1_chains(rho):
    """An AR(1) chain with coefficient rho has integrated autocorrelation time (1 + rho) / (1 - rho)."""
    n = 40000
    expect = n * (1 - rho) / (1 + rho)
    got = np.mean([hmc.ess(ar1(n, rho, s)) for s in range(4)])
    assert abs(got - expect) <= 0.12 * expect


def test_leapfrog_is_reversible():
    rng = np.random.default_rng(1)
    g = Gaussian(rng.normal(size=6), rng.uniform(0.3, 3.0, size=6))
    minv = rng.uniform(0.5, 2.0, size=6)
    th0, p0 = rng.normal(size=6), rng.normal(size=6)
    _, grad0 = g.logp_grad(th0)
    th1, p1, _, grad1 = hmc.leapfrog(th0, p0, grad0, 0.05, 40, minv, g.logp_grad)
    th2, p2, _, _ = hmc.leapfrog(th1, -p1, grad1, 0.05, 40, minv, g.logp_grad)
    np.testing.assert_allclose(th2, th0, atol=1e-11)
    np.testing.assert_allclose(-p2, p0, atol=1e-11)


def test_leapfrog_energy_error_is_second_order():
    """Over a fixed trajectory length, halving the step divides the energy error by about 4."""
    rng = np.random.default_rng(2)
    g = Gaussian(np.zeros(5), np.array([0.5, 1.0, 1.5, 2.0, 3.0]))
    minv = np.ones(5)

    def mean_abs_dh(eps, n):
        out = []
        for s in range(30):
            r = np.random.default_rng(100 + s)
            th, p = r.normal(size=5), r.normal(size=5)
            lp, gr = g.logp_grad(th)
            th1, p1, lp1, _ = hmc.leapfrog(th, p, gr, eps, n, minv, g.logp_grad)
            out.append(abs((-lp1 + 0.5 * p1 @ p1) - (-lp + 0.5 * p @ p)))
        return np.mean(out)

    ratio = mean_abs_dh(0.1, 20) / mean_abs_dh(0.05, 40)
    assert 3.0 < ratio < 5.5


def test_adaptive_mass_samples_an_anisotropic_gaussian():
    mean, sd = np.array([1.0, -2.0, 3.0, 0.0]), np.array([0.05, 1.0, 20.0, 3.0])
    g = Gaussian(mean, sd)
    r = hmc.hmc(g, mean + sd, n_iter=4000, eps=0.01, n_leapfrog=8, adapt_mass=True, k=10,
                adapt_eps_until=500, seed=3)
    # the Hessian diagonal is constant, so after the first update the mass is the precision
    np.testing.assert_allclose(r["mass"], 1.0 / sd ** 2, rtol=1e-12)
    x = r["samples"][1000:]
    for i in range(4):
        n_eff = hmc.ess(x[:, i])
        assert n_eff > 200
        assert abs(x[:, i].mean() - mean[i]) < 5 * sd[i] / np.sqrt(n_eff)
        assert abs(x[:, i].std() / sd[i] - 1.0) < 0.15
    assert 0.5 < r["accepted"][1000:].mean() <= 1.0


def test_mass_update_is_the_clamped_running_mean():
    class Counting(Gaussian):
        def __init__(self):
            super().__init__(np.zeros(3), np.ones(3))
            self.calls = 0

        def neg_hess_diag(self, th):
            self.calls += 1
            return np.array([float(self.calls), 1e9, 1e-9])

    g = Counting()
    r = hmc.hmc(g, np.zeros(3), n_iter=30, eps=0.1, n_leapfrog=2, k=10, m_min=1e-3, m_max=1e6, seed=4)
    assert g.calls == 3   # iterations 10, 20, 30
    np.testing.assert_allclose(r["mass"], [2.0, 1e6, 1e-3])
    r = hmc.hmc(g, np.zeros(3), n_iter=30, eps=0.1, n_leapfrog=2, adapt_mass=False, seed=4)
    np.testing.assert_array_equal(r["mass"], np.ones(3))
    assert r["gradient_evaluations"] == 1 + 30 * 2
