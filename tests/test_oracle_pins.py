"""Pins of the FP64 oracle against things fixed by the paper and by mathematics, not by itself.

* expm: scipy's independent implementation, the JC69 and 2-state closed forms, the semigroup
  property.
* likelihood: the definition Eq. 1 summed by brute force over internal states (with the rate
  mixture of Section 2.5), 2-taxon and zero-length closed forms, an underflow closed form.
* gradient: term-by-term derivative of Eq. 1, the quadratic pruning gradient (Section 1),
  central finite differences, the pulley principle.
* pre-order partials: p_k' q_k = P(Y) at every node (Section 2.4).
* invariances: root position for reversible stationary Q (Section 5), Q*c with b/c,
  identical rate categories, internal relabelling.
* Hessian diagonal (Section 2.6): finite differences of the gradient; the exact derivatives of
  the closed-form 2-state transition matrices.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1905_12146_gb300 import workloads as wl
from tests import independent as ind


def _tiny(n_tips, seed, n_cat=2, n_pat=40, ambiguous=0.15, n_models=1, m=4):
    pr = wl.random_problem(n_tips, n_pat, n_states=m, n_cat=n_cat, seed=seed, b_mean=0.3,
                           ambiguous=ambiguous, weights="int", n_models=n_models)
    return pr


# ------------------------------------------------------------------------------ expm


@pytest.mark.parametrize("m", [2, 4, 20, 61])
def test_expm_matches_scipy(oracle_mod, m):
    rng = np.random.default_rng(m)
    for scale in (1e-3, 0.3, 2.0, 40.0):
        A = rng.normal(size=(m, m)) * scale / np.sqrt(m)
        ref = sla.expm(A)
        got = oracle_mod.expm(A)
        assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_expm_jc69_closed_form(oracle_mod):
    Q = wl.jc69_Q()
    for t in (0.0, 1e-4, 0.05, 0.7, 3.0, 25.0):
        P = oracle_mod.expm(Q * t)
        e = np.exp(-4.0 * t / 3.0)
        ref = np.full((4, 4), 0.25 - 0.25 * e)
        np.fill_diagonal(ref, 0.25 + 0.75 * e)
        assert np.abs(P - ref).max() < 5e-14


def test_expm_semigroup_and_stochastic(oracle_mod):
    rng = np.random.default_rng(7)
    for m in (4, 61):
        Q = wl.random_general_Q(m, rng) if m == 4 else wl.codon_Q(rng)[0]
        s, t = 0.13, 0.41
        Ps, Pt, Pst = (oracle_mod.expm(Q * x) for x in (s, t, s + t))
        assert np.abs(Ps @ Pt - Pst).max() < 1e-13
        assert np.abs(Pst.sum(axis=1) - 1.0).max() < 1e-13
        assert Pst.min() >= -1e-15


# ------------------------------------------------------------------------------ likelihood


@pytest.mark.parametrize("n_tips,seed,n_models", [(2, 0, 1), (3, 1, 1), (4, 2, 2), (5, 3, 1),
                                                   (6, 4, 3)])
def test_loglik_and_gradient_brute_force(oracle_mod, n_tips, seed, n_models):
    pr = _tiny(n_tips, seed, n_models=n_models)
    L, dL = ind.brute_force(pr)
    r = oracle_mod.evaluate(pr)
    np.testing.assert_allclose(r.site_logL, np.log(L), rtol=1e-12, atol=1e-12)
    w = pr["weights"]
    assert abs(r.logL - np.sum(w * np.log(L))) <= 1e-12 * abs(r.logL)
    g_ref = (w[None, :] * dL / L[None, :]).sum(axis=1)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_two_taxon_closed_form(oracle_mod):
    rng = np.random.default_rng(11)
    Q = wl.random_general_Q(4, rng)
    pi = wl.dirichlet_freqs(4, rng)
    parent = np.array([2, 2, -1], dtype=np.int32)
    tips = np.array([[0, 1, 2, 3, 4, 1], [0, 3, 2, 4, 4, 0]], dtype=np.uint8)
    b = np.array([0.3, 0.07, 0.0])
    pr = wl.make_problem(parent, tips, np.ones(6), Q, pi, np.ones(1), np.ones(1), b)
    P1, P2 = sla.expm(Q * b[0]), sla.expm(Q * b[1])
    ones = np.ones(4)
    ref = []
    for y1, y2 in tips.T:
        v1 = P1 @ (ones if y1 >= 4 else np.eye(4)[y1])
        v2 = P2 @ (ones if y2 >= 4 else np.eye(4)[y2])
        ref.append(np.log(np.sum(pi * v1 * v2)))
    np.testing.assert_allclose(oracle_mod.evaluate(pr).site_logL, ref, rtol=1e-13, atol=1e-14)


def test_zero_branch_lengths_closed_form(oracle_mod):
    """b = 0 gives P = I: a site is possible only if all observed tips agree, L = pi_state."""
    rng = np.random.default_rng(12)
    parent, _ = wl.yule_tree(9, rng)
    pi = wl.dirichlet_freqs(4, rng)
    states = rng.integers(0, 4, size=30)
    tips = np.repeat(states[None, :], 9, axis=0).astype(np.uint8)
    tips[rng.random(tips.shape) < 0.3] = 4
    pr = wl.make_problem(parent, tips, np.ones(30), wl.random_general_Q(4, rng), pi,
                         np.ones(1), np.ones(1), np.zeros(parent.shape[0]))
    np.testing.assert_allclose(oracle_mod.evaluate(pr).site_logL, np.log(pi[states]), rtol=1e-14)


def test_underflow_closed_form(oracle_mod):
    """JC69 with every tip branch saturated (b=60): L_p = 4^-N exactly; N=700 gives 2^-1400,
    far below the FP64 range, so this exercises the power-of-two rescaling."""
    n_tips = 700
    rng = np.random.default_rng(13)
    parent, _ = wl.yule_tree(n_tips, rng)
    b = rng.exponential(0.1, size=parent.shape[0])
    b[:n_tips] = 60.0
    b[parent < 0] = 0.0
    tips = rng.integers(0, 5, size=(n_tips, 8)).astype(np.uint8)
    pr = wl.make_problem(parent, tips, np.ones(8), wl.jc69_Q(), np.full(4, 0.25), np.ones(1),
                         np.ones(1), b)
    site = oracle_mod.evaluate(pr).site_logL
    n_obs = (tips < 4).sum(axis=0)
    np.testing.assert_allclose(site, -n_obs * np.log(4.0), rtol=1e-12)


# ------------------------------------------------------------------------------ gradient


def test_gradient_quadratic_pruning(oracle_mod):
    pr = wl.random_problem(14, 60, n_states=4, n_cat=3, seed=21, b_mean=0.2, ambiguous=0.1,
                           weights="int", n_models=3)
    g_ref, logL_ref = ind.quadratic_gradient(pr)
    r = oracle_mod.evaluate(pr)
    assert abs(r.logL - logL_ref) <= 1e-12 * abs(logL_ref)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_gradient_quadratic_pruning_codon(oracle_mod):
    pr = wl.random_problem(5, 12, n_states=61, n_cat=2, seed=22, b_mean=0.2)
    g_ref, logL_ref = ind.quadratic_gradient(pr)
    r = oracle_mod.evaluate(pr)
    assert abs(r.logL - logL_ref) <= 1e-11 * abs(logL_ref)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-9, atol=1e-9 * np.abs(g_ref).max())


def test_gradient_central_differences(oracle_mod):
    pr = wl.config_small(seed=0)
    r = oracle_mod.evaluate(pr)
    h = 1e-6
    b = pr["b"]
    fd = np.zeros_like(b)
    for i in range(b.shape[0]):
        if pr["parent"][i] < 0:
            continue
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd[i] = (oracle_mod.evaluate(pr, bp).logL - oracle_mod.evaluate(pr, bm).logL) / (2 * h)
    assert np.abs(fd - r.grad).max() <= 1e-5 * np.abs(r.grad).max()


def test_hessian_diagonal_central_differences(oracle_mod):
    pr = wl.random_problem(12, 200, n_states=4, n_cat=3, seed=23, b_mean=0.1, ambiguous=0.05,
                           weights="int")
    r = oracle_mod.evaluate(pr)
    h = 1e-5
    b = pr["b"]
    for i in range(b.shape[0]):
        if pr["parent"][i] < 0:
            assert r.hess[i] == 0.0
            continue
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle_mod.evaluate(pr, bp).grad[i] - oracle_mod.evaluate(pr, bm).grad[i]) / (2 * h)
        assert abs(fd - r.hess[i]) <= 1e-5 * max(1.0, abs(r.hess[i]))


def test_two_state_closed_form_gradient_and_hessian(oracle_mod):
    """A non-reversible 2-state chain Q = [[-a, a], [c, -c]] has, with s = a + c and E = e^-st,
    P(t) = ([[c, a], [c, a]] + E [[a, -a], [-c, c]]) / s, so dP/dt = E Q and d2P/dt2 = -s E Q.
    On a 3-taxon tree with a non-stationary root distribution and two unequally weighted rate
    categories, Eq. 1 is summed over the internal states with these matrices; differentiating one
    branch's factor once or twice gives the gradient and the Hessian diagonal exactly (Section
    2.6, summed over sites with the per-site squared gradient)."""
    a, c = 0.7, 1.9
    s_ = a + c
    Q = np.array([[-a, a], [c, -c]])

    def P(t, k):
        E = np.exp(-s_ * t)
        if k == 0:
            return (np.array([[c, a], [c, a]]) + E * np.array([[a, -a], [-c, c]])) / s_
        return (E if k == 1 else -s_ * E) * Q

    parent = np.array([3, 3, 4, 4, -1], dtype=np.int32)
    tips = np.array([[0, 1, 0, 2, 1, 0, 2], [0, 0, 1, 1, 2, 1, 0], [1, 0, 0, 1, 0, 2, 1]], dtype=np.uint8)
    wt = np.array([3.0, 1.0, 2.0, 1.0, 5.0, 1.0, 2.0])
    pi = np.array([0.8, 0.2])
    rates, cw = np.array([0.4, 1.9]), np.array([0.65, 0.35])
    b = np.array([0.3, 0.05, 0.9, 0.2, 0.0])
    pr = wl.make_problem(parent, tips, wt, Q, pi, rates, cw, b)

    def tip(y):
        return np.ones(2) if y >= 2 else np.eye(2)[y]

    def L(p, branch=-1, k=0):
        """L_p, or its k-th derivative in b_branch."""
        tot = 0.0
        for r, w in zip(rates, cw):
            M = {i: P(r * b[i], 0) for i in range(4)}
            if branch >= 0:
                M[branch] = r ** k * P(r * b[branch], k)
            v3 = (M[0] @ tip(tips[0, p])) * (M[1] @ tip(tips[1, p]))
            tot += w * pi @ ((M[3] @ v3) * (M[2] @ tip(tips[2, p])))
        return tot

    n_pat = tips.shape[1]
    logL = sum(wt[p] * np.log(L(p)) for p in range(n_pat))
    grad, hess = np.zeros(5), np.zeros(5)
    for i in range(4):
        for p in range(n_pat):
            g = L(p, i, 1) / L(p)
            grad[i] += wt[p] * g
            hess[i] += wt[p] * (L(p, i, 2) / L(p) - g * g)
    r = oracle_mod.evaluate(pr)
    assert abs(r.logL - logL) <= 1e-13 * abs(logL)
    np.testing.assert_allclose(r.grad, grad, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(r.hess, hess, rtol=1e-11, atol=1e-13)


# ------------------------------------------------------------------------------ partials


def test_pre_post_inner_product_at_every_node(oracle_mod):
    """P(Y) = sum_l w_l p_k,l' q_k,l for every node k (Section 2.4 and the mixture of 2.5)."""
    pr = wl.random_problem(25, 50, n_states=4, n_cat=3, seed=31, b_mean=0.1, ambiguous=0.1)
    r = oracle_mod.evaluate(pr, partials=True)
    cw = pr["cat_weights"]
    for k in range(pr["parent"].shape[0]):
        inner = np.einsum("pls,pls,l->p", r.post[k], r.pre[k], cw)
        logs = np.log(inner) + (r.post_e[k] + r.pre_e[k]) * np.log(2.0)
        np.testing.assert_allclose(logs, r.site_logL, rtol=1e-13, atol=1e-12)


def test_root_pre_order_partial_is_pi(oracle_mod):
    pr = wl.random_problem(7, 10, n_states=4, n_cat=2, seed=32)
    r = oracle_mod.evaluate(pr, partials=True)
    root = wl.root_of(pr["parent"])
    assert np.all(r.pre_e[root] == 0)
    np.testing.assert_array_equal(r.pre[root], np.broadcast_to(pr["root_freqs"], r.pre[root].shape))


# ------------------------------------------------------------------------------ invariances


def test_root_position_invariance_reversible(oracle_mod):
    pr = wl.random_problem(10, 80, n_states=4, n_cat=2, seed=41, b_mean=0.2, reversible=True,
                           ambiguous=0.05)
    base = oracle_mod.evaluate(pr)
    rng = np.random.default_rng(0)
    for edge in rng.choice(np.flatnonzero(pr["parent"] >= 0), size=5, replace=False):
        par2, b2 = ind.reroot(pr["parent"], pr["b"], int(edge), float(rng.uniform(0.1, 0.9)))
        pr2 = dict(pr, parent=par2, b=b2)
        assert abs(oracle_mod.evaluate(pr2).logL - base.logL) <= 1e-12 * abs(base.logL)
    # pulley principle: the two root branches share one derivative
    root = wl.root_of(pr["parent"])
    a, c = np.flatnonzero(pr["parent"] == root)
    assert abs(base.grad[a] - base.grad[c]) <= 1e-10 * np.abs(base.grad).max()


def test_root_position_matters_when_nonreversible(oracle_mod):
    """Section 5: rerooting invariance needs reversibility; a general Q breaks it."""
    pr = wl.random_problem(10, 80, n_states=4, n_cat=1, seed=42, b_mean=0.3)
    base = oracle_mod.evaluate(pr).logL
    par2, b2 = ind.reroot(pr["parent"], pr["b"], 0, 0.5)
    assert abs(oracle_mod.evaluate(dict(pr, parent=par2, b=b2)).logL - base) > 1e-6


def test_time_rescaling(oracle_mod):
    pr = wl.random_problem(12, 40, n_states=4, n_cat=2, seed=51, ambiguous=0.1)
    r = oracle_mod.evaluate(pr)
    c = 2.5
    r2 = oracle_mod.evaluate(dict(pr, Q=pr["Q"] * c), pr["b"] / c)
    assert abs(r2.logL - r.logL) <= 1e-12 * abs(r.logL)
    np.testing.assert_allclose(r2.grad, r.grad * c, rtol=1e-10, atol=1e-10 * np.abs(r.grad).max())


def test_identical_categories_equal_single_category(oracle_mod):
    pr = wl.random_problem(12, 40, n_states=4, n_cat=1, seed=52, ambiguous=0.1)
    r1 = oracle_mod.evaluate(pr)
    pr3 = dict(pr, cat_rates=np.ones(3), cat_weights=np.array([0.2, 0.5, 0.3]))
    r3 = oracle_mod.evaluate(pr3)
    assert abs(r3.logL - r1.logL) <= 1e-13 * abs(r1.logL)
    np.testing.assert_allclose(r3.grad, r1.grad, rtol=1e-12, atol=1e-12 * np.abs(r1.grad).max())


def test_internal_relabelling_invariance(oracle_mod):
    pr = wl.random_problem(30, 40, n_states=4, n_cat=2, seed=53, ambiguous=0.1)
    r = oracle_mod.evaluate(pr)
    par2, perm = wl.relabel_nodes(pr["parent"], np.random.default_rng(1), 30)
    b2 = np.zeros_like(pr["b"])
    b2[perm] = pr["b"]
    r2 = oracle_mod.evaluate(dict(pr, parent=par2), b2)
    assert abs(r2.logL - r.logL) <= 1e-12 * abs(r.logL)
    np.testing.assert_allclose(r2.grad[perm], r.grad, rtol=1e-11, atol=1e-12)


def test_rejects_malformed_trees(oracle_mod):
    pr = wl.random_problem(6, 5, seed=54)
    bad = pr["parent"].copy()
    bad[wl.root_of(bad)] = 0          # no root (a cycle)
    with pytest.raises(ValueError):
        oracle_mod.evaluate(dict(pr, parent=bad))
    bad = pr["parent"].copy()
    bad[0] = bad[1] = bad[2] = bad[3]  # 2N-1 nodes with a node of degree > 2: another has < 2 children
    with pytest.raises(ValueError):
        oracle_mod.evaluate(dict(pr, parent=bad))
    with pytest.raises(ValueError):
        oracle_mod.evaluate(pr, -pr["b"] - 0.1)
