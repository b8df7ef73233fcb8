"""Pins of the oracle on trees with multifurcations (internal nodes with more than two children).

The paper's tree is binary (Section 2.1).  With a wider sibling set the post-order update takes the
product of P_c p_c over all children c and the pre-order update multiplies q_k by P_s p_s over every
sibling s of the updated child (Sections 2.3-2.4 with the sibling set widened).  Pinned, without the
oracle's code, by:

- brute force over every internal-state assignment (Eq. 1 with the rate mixture of Section 2.5), and
  its term-by-term derivative, on 5- and 6-taxon trees with nodes of degree 3 and 4 and a star tree;
- the quadratic "substitute dP for P and prune again" gradient on a larger tree;
- the binary tree obtained by splitting each multifurcation with branches of length 0 (their
  transition matrices are the identity, so likelihood and the derivatives in every original branch
  are unchanged), built independently of the oracle and of the library;
- central differences of the gradient for the Hessian diagonal.
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl
from tests import independent as ind


def _problem(parent, n_tips, seed, n_pat=30, m=4, n_cat=2, b_mean=0.3, ambiguous=0.15):
    """Data and model of random_problem on a given (multifurcating) topology."""
    base = wl.random_problem(n_tips, n_pat, n_states=m, n_cat=n_cat, seed=seed, b_mean=b_mean,
                             ambiguous=ambiguous, weights="int")
    rng = np.random.default_rng(seed + 77)
    parent = np.asarray(parent, dtype=np.int32)
    b = rng.exponential(b_mean, size=parent.shape[0])
    b[parent < 0] = 0.0
    return dict(base, parent=parent, b=b, n_tips=n_tips, node_time=None, branch_model=None)


# 5 taxa, two trifurcations: root 5 -> (0, 4, 6), 6 -> (1, 2, 3)
FIVE_TWO_TRIFURCATIONS = ([5, 6, 6, 6, 5, -1, 5], 5)
# 5 taxa with one trifurcation: 5 -> (6, 7); 6 -> (0, 1, 2); 7 -> (3, 4)
FIVE_ONE_TRIFURCATION = ([6, 6, 6, 7, 7, -1, 5, 5], 5)
# star tree: the root holds all four tips
STAR4 = ([4, 4, 4, 4, -1], 4)
# 6 taxa: 6 -> (0, 7); 7 -> (1, 2, 3, 8) (degree 4); 8 -> (4, 5)
SIX_DEGREE_FOUR = ([6, 7, 7, 7, 8, 8, -1, 6, 7], 6)


@pytest.mark.parametrize("tree,seed", [(FIVE_ONE_TRIFURCATION, 1), (FIVE_TWO_TRIFURCATIONS, 2), (STAR4, 3),
                                       (SIX_DEGREE_FOUR, 4)])
def test_multifurcation_brute_force(oracle_mod, tree, seed):
    pr = _problem(*tree, seed)
    L, dL = ind.brute_force(pr)
    r = oracle_mod.evaluate(pr)
    np.testing.assert_allclose(r.site_logL, np.log(L), rtol=1e-12, atol=1e-12)
    w = pr["weights"]
    assert abs(r.logL - np.sum(w * np.log(L))) <= 1e-12 * abs(r.logL)
    g_ref = (w[None, :] * dL / L[None, :]).sum(axis=1)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_multifurcation_brute_force_three_states_general_model(oracle_mod):
    """A non-reversible 3-state generator and a root distribution that is not stationary."""
    pr = _problem(*SIX_DEGREE_FOUR, seed=5, m=3)
    rng = np.random.default_rng(5)
    pr["Q"] = wl.random_general_Q(3, rng)[None]
    pr["root_freqs"] = wl.dirichlet_freqs(3, rng)
    L, dL = ind.brute_force(pr)
    r = oracle_mod.evaluate(pr)
    np.testing.assert_allclose(r.site_logL, np.log(L), rtol=1e-12, atol=1e-12)
    g_ref = (pr["weights"][None, :] * dL / L[None, :]).sum(axis=1)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_multifurcation_quadratic_gradient(oracle_mod):
    pr = wl.multifurcating_problem(20, 60, 6, n_states=4, n_cat=3, seed=6, b_mean=0.1, ambiguous=0.05)
    assert np.bincount(pr["parent"][pr["parent"] >= 0]).max() >= 3
    g, ll = ind.quadratic_gradient(pr)
    r = oracle_mod.evaluate(pr)
    assert abs(r.logL - ll) <= 1e-12 * abs(ll)
    np.testing.assert_allclose(r.grad, g, rtol=1e-10, atol=1e-10 * np.abs(g).max())


@pytest.mark.parametrize("m,n_collapse,seed", [(4, 5, 7), (20, 3, 8), (61, 2, 9)])
def test_multifurcation_equals_zero_length_resolution(oracle_mod, m, n_collapse, seed):
    """The multifurcating tree and its binary resolution with zero-length branches give the same
    site likelihoods, and the same gradient and Hessian diagonal in every original branch."""
    pr = wl.multifurcating_problem(16, 40, n_collapse, n_states=m, n_cat=2, seed=seed, b_mean=0.1, ambiguous=0.05)
    rb, n = ind.resolve_zero_length(pr)
    a = oracle_mod.evaluate(pr)
    c = oracle_mod.evaluate(rb)
    np.testing.assert_allclose(a.site_logL, c.site_logL, rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(a.grad, c.grad[:n], rtol=1e-11, atol=1e-11 * np.abs(a.grad).max())
    np.testing.assert_allclose(a.hess, c.hess[:n], rtol=1e-10, atol=1e-10 * np.abs(a.hess).max())


def test_multifurcation_hessian_central_differences(oracle_mod):
    pr = wl.multifurcating_problem(10, 50, 3, n_states=4, n_cat=2, seed=10, b_mean=0.2, ambiguous=0.05)
    r = oracle_mod.evaluate(pr)
    root = wl.root_of(pr["parent"])
    for i in range(pr["parent"].shape[0]):
        if i == root:
            continue
        h = 1e-5 * max(pr["b"][i], 1e-3)
        bp, bm = pr["b"].copy(), pr["b"].copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle_mod.evaluate(pr, bp).grad[i] - oracle_mod.evaluate(pr, bm).grad[i]) / (2 * h)
        assert abs(fd - r.hess[i]) <= 1e-5 * max(1.0, abs(r.hess[i]))


def test_multifurcation_rejections(oracle_mod):
    pr = _problem(*FIVE_ONE_TRIFURCATION, seed=11)
    bad = pr["parent"].copy()
    bad[4] = 6                       # node 7 keeps one child
    with pytest.raises(ValueError):
        oracle_mod.evaluate(dict(pr, parent=bad))
    bad = pr["parent"].copy()
    bad[3] = 2                       # a tip with a child
    with pytest.raises(ValueError):
        oracle_mod.evaluate(dict(pr, parent=bad))
