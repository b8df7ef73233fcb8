"""Hamiltonian Monte Carlo for branch-specific evolutionary rates (Section 3.2), with the diagonal
mass matrix adapted to the posterior-averaged Hessian diagonal (Section 3.2.1).

Target (Section 4.2, random-effects relaxed clock, with the tree-wise mean mu and the scale psi
held fixed): branch i evolves at r_i = mu eps_i for its duration dt_i = t_i - t_parent(i), so
b_i = r_i dt_i.  The random effects are lognormal with mean 1 and variance psi^2, i.e.
theta_i = log eps_i ~ N(-s2 / 2, s2) with s2 = log(1 + psi^2), and

    log pi(theta) = logL(b(theta)) + sum_i log N(theta_i; -s2 / 2, s2).

One library evaluation gives logL, its gradient g and Hessian diagonal h in b (post-order and
pre-order passes, Sections 2.3-2.5; the diagonal Hessian of the Appendix).  With d b_i / d theta_i
= b_i the chain rule gives

    d logL / d theta_i = b_i g_i,        d^2 logL / d theta_i^2 = b_i g_i + b_i^2 h_i.

The sampler (``hmc``) works on any target with ``logp_grad(theta) -> (log pi, gradient)`` and,
for the adaptive mass matrix, ``neg_hess_diag(theta)``.  Leapfrog integration, the Metropolis
test, and the mass matrix follow Section 3.2.  The mass matrix update runs every k = 10
iterations.  It sets M_ii to the running mean of -d^2 log pi / d theta_i^2 over the update points,
clamped to [m_min, m_max].
"""
from __future__ import annotations

import math
import time

import numpy as np


class ClockTarget:
    """log pi(theta) of the random-effects clock on the problem in ``handle`` (one tree).

    ``node_times`` [2N-1] in forward time.  theta holds one entry per non-root node, in node order
    (``self.nodes``).  Evaluations go through ``handle.eval`` (host arrays); use an FP64 handle so
    that the Metropolis test sees logL to double precision."""

    def __init__(self, handle, parent, node_times, mu: float, psi: float):
        parent = np.asarray(parent)
        t = np.asarray(node_times, dtype=np.float64)
        self.handle = handle
        self.nodes = np.flatnonzero(parent >= 0)
        self.dt = t[self.nodes] - t[parent[self.nodes]]
        if np.any(self.dt <= 0):
            raise ValueError("every branch needs t_i > t_parent(i)")
        self.mu = float(mu)
        self.s2 = math.log1p(float(psi) ** 2)
        self.m = -0.5 * self.s2
        self.n_nodes = parent.shape[0]
        self.evaluations = 0

    @property
    def dim(self) -> int:
        return self.nodes.shape[0]

    def _b(self, theta):
        b = np.zeros(self.n_nodes)
        b[self.nodes] = self.mu * np.exp(theta) * self.dt
        return b

    def _eval(self, theta, hess: bool):
        b = self._b(theta)
        r = self.handle.eval(b, grad=True, hess=hess)
        self.evaluations += 1
        if r["status"] != 0:
            raise RuntimeError(f"likelihood evaluation failed with status {r['status']}")
        return r, b[self.nodes]

    def logp_grad(self, theta):
        r, bn = self._eval(theta, False)
        d = theta - self.m
        logp = r["logL"] - 0.5 * float(d @ d) / self.s2 - 0.5 * theta.size * math.log(2 * math.pi * self.s2)
        grad = bn * r["grad"][self.nodes] - d / self.s2
        return logp, grad

    def neg_hess_diag(self, theta):
        r, bn = self._eval(theta, True)
        g, h = r["grad"][self.nodes], r["hess"][self.nodes]
        return -(bn * g + bn * bn * h) + 1.0 / self.s2


def leapfrog(theta, p, grad, eps: float, n: int, minv, logp_grad):
    """n leapfrog steps of size eps from (theta, p) with the gradient at theta given (Section 3.2):
    half kick, drift by M^-1 p, half kick.  Returns (theta, p, log pi, gradient) at the end."""
    theta = theta.copy()
    p = p + 0.5 * eps * grad
    logp = None
    for i in range(n):
        theta = theta + eps * minv * p
        logp, grad = logp_grad(theta)
        if not np.isfinite(logp):
            return theta, p, -np.inf, grad
        p = p + (eps if i + 1 < n else 0.5 * eps) * grad
    return theta, p, logp, grad


def hmc(target, theta0, n_iter: int, eps: float, n_leapfrog: int, adapt_mass: bool = True, k: int = 10,
        m_min: float = 1e-3, m_max: float = 1e6, adapt_eps_until: int = 0, target_accept: float = 0.8,
        seed: int = 0):
    """Run n_iter HMC iterations from theta0.

    Mass matrix: the identity until the first update.  With ``adapt_mass`` the update happens at
    every iteration s that is a multiple of k.  It evaluates -d^2 log pi / d theta^2 at theta^(s),
    keeps the running mean H over these points, and uses M = clip(H, m_min, m_max) from iteration
    s + 1 on.  Step size: fixed, unless ``adapt_eps_until`` > 0.  Then, up to that iteration, eps
    is scaled by exp(0.1 (accept - target_accept)) after every iteration.  This is a warm-up aid,
    and the samples drawn while eps is still adapting should be discarded.

    Returns a dict with the samples [n_iter, dim], the acceptance indicators, the final eps and
    mass diagonal, the number of gradient evaluations and the wall seconds."""
    rng = np.random.default_rng(seed)
    theta = np.asarray(theta0, dtype=np.float64).copy()
    d = theta.size
    mass = np.ones(d)
    hsum = np.zeros(d)
    n_upd = 0
    logp, grad = target.logp_grad(theta)
    n_grad = 1
    samples = np.empty((n_iter, d))
    accepted = np.zeros(n_iter, dtype=bool)
    t0 = time.perf_counter()
    for s in range(1, n_iter + 1):
        p0 = rng.standard_normal(d) * np.sqrt(mass)
        minv = 1.0 / mass
        th1, p1, logp1, grad1 = leapfrog(theta, p0, grad, eps, n_leapfrog, minv, target.logp_grad)
        n_grad += n_leapfrog
        h0 = -logp + 0.5 * float(p0 @ (minv * p0))
        h1 = -logp1 + 0.5 * float(p1 @ (minv * p1)) if np.isfinite(logp1) else np.inf
        log_a = min(0.0, h0 - h1)
        acc = bool(np.log(rng.random()) < log_a)
        if acc:
            theta, logp, grad = th1, logp1, grad1
        samples[s - 1] = theta
        accepted[s - 1] = acc
        if s <= adapt_eps_until:
            eps *= math.exp(0.1 * (math.exp(log_a) - target_accept))
        if adapt_mass and s % k == 0:
            hsum += target.neg_hess_diag(theta)
            n_upd += 1
            mass = np.clip(hsum / n_upd, m_min, m_max)
    return {"samples": samples, "accepted": accepted, "eps": eps, "mass": mass, "gradient_evaluations": n_grad,
            "seconds": time.perf_counter() - t0}


def ess(x) -> float:
    """Effective sample size of a 1-D chain: n / tau with tau = -1 + 2 sum_k Gamma_k, Gamma_k =
    rho_2k + rho_2k+1 summed while positive and made monotone (Geyer's initial monotone sequence
    estimator, Statistical Science 1992).  Antithetic chains can give tau < 1.  tau is bounded below
    by 1 / log10(n), so the ESS is at most n log10(n), the cap Stan uses."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    if n < 4:
        return float(n)
    y = x - x.mean()
    var = float(y @ y) / n
    if var == 0.0:
        return float(n)
    f = np.fft.rfft(y, 2 * n)
    acov = np.fft.irfft(f * np.conj(f))[:n] / n
    rho = acov / var
    tau = -1.0
    prev = np.inf
    for j in range(0, n - 1, 2):
        g = rho[j] + rho[j + 1]
        if g <= 0.0:
            break
        g = min(g, prev)
        tau += 2.0 * g
        prev = g
    return n / max(tau, 1.0 / math.log10(n))
