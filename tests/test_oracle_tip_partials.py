"""Pins of the oracle for partially observed tips (Section 2.1: a tip's post-order partial vector
may carry partial observations or missing data instead of the indicator of one state).

A code m + k selects row k of a per-problem table of partial vectors; codes past the table are
missing data.  The pins do not go through the oracle's code for these vectors:

* brute force over internal states (Eq. 1), each tip factor summed over the tip's states with its
  partial vector as weights, for logL and, term by term, the gradient;
* the quadratic "substitute dP for P and prune again" gradient (Section 1) on a larger tree;
* linearity: a site's likelihood is linear in a tip's partial vector, so with vector v it equals
  sum_j v_j times the likelihood of the same site with that tip observed in state j;
* central differences of the gradient for the Hessian diagonal (Section 2.6);
* special rows: an indicator row equals the plain state code and an all-ones row equals missing
  data, bit for bit.
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl
from tests import independent as ind


def _partial_problem(n_tips, n_pat, seed, m=4, n_cat=2, frac=0.3, b_mean=0.3, n_models=1):
    pr = wl.random_problem(n_tips, n_pat, n_states=m, n_cat=n_cat, seed=seed, b_mean=b_mean,
                           ambiguous=0.1, weights="int", n_models=n_models)
    rng = np.random.default_rng(seed + 1000)
    if m == 4:
        table = wl.iupac_nucleotide_partials(error=0.03)
    else:   # random subsets and graded rows
        table = np.where(rng.random((12, m)) < 0.3, rng.uniform(0.2, 1.0, (12, m)), 0.0)
        table[np.arange(12), rng.integers(0, m, 12)] = 1.0
    pr["tip_partials"] = table
    pr["tip_states"] = wl.make_partially_observed(pr["tip_states"], frac, table, rng)
    return pr


@pytest.mark.parametrize("n_tips,seed,n_models", [(3, 1, 1), (4, 2, 2), (5, 3, 1)])
def test_brute_force(oracle_mod, n_tips, seed, n_models):
    pr = _partial_problem(n_tips, 50, seed, n_models=n_models)
    assert (pr["tip_states"] >= 4).any() and (pr["tip_states"] < wl.MISSING).any()
    L, dL = ind.brute_force(pr)
    r = oracle_mod.evaluate(pr)
    np.testing.assert_allclose(r.site_logL, np.log(L), rtol=1e-12, atol=1e-12)
    w = pr["weights"]
    g_ref = (w[None, :] * dL / L[None, :]).sum(axis=1)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_brute_force_general_state_space(oracle_mod):
    pr = _partial_problem(3, 30, 7, m=6, n_cat=1)
    L, dL = ind.brute_force(pr)
    r = oracle_mod.evaluate(pr)
    np.testing.assert_allclose(r.site_logL, np.log(L), rtol=1e-12, atol=1e-12)
    g_ref = (pr["weights"][None, :] * dL / L[None, :]).sum(axis=1)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_quadratic_gradient(oracle_mod):
    pr = _partial_problem(14, 60, 21, n_cat=3, n_models=2, b_mean=0.2)
    g_ref, logL_ref = ind.quadratic_gradient(pr)
    r = oracle_mod.evaluate(pr)
    assert abs(r.logL - logL_ref) <= 1e-12 * abs(logL_ref)
    np.testing.assert_allclose(r.grad, g_ref, rtol=1e-10, atol=1e-10 * np.abs(g_ref).max())


def test_likelihood_is_linear_in_a_tip_vector(oracle_mod):
    """One tip with a partial vector v at every site, the other tips observed: L(v) = sum_j v_j L(e_j)."""
    m = 4
    pr = wl.random_problem(20, 40, n_states=m, n_cat=2, seed=31, b_mean=0.1)
    rng = np.random.default_rng(31)
    table = rng.uniform(0.0, 1.0, (5, m))
    table[rng.random((5, m)) < 0.3] = 0.0
    table[:, 0] += 0.1
    t = 7
    codes = rng.integers(0, 5, size=40)
    pr_v = dict(pr, tip_partials=table, tip_states=pr["tip_states"].copy())
    pr_v["tip_states"][t] = m + codes
    site_v = oracle_mod.evaluate(pr_v).site_logL
    site_j = []
    for j in range(m):
        pj = dict(pr, tip_states=pr["tip_states"].copy())
        pj["tip_states"][t] = j
        site_j.append(oracle_mod.evaluate(pj).site_logL)
    ref = np.log(sum(table[codes, j] * np.exp(site_j[j]) for j in range(m)))
    np.testing.assert_allclose(site_v, ref, rtol=1e-12)


def test_hessian_diagonal_central_differences(oracle_mod):
    pr = _partial_problem(10, 120, 23, n_cat=3, b_mean=0.1)
    r = oracle_mod.evaluate(pr)
    h = 1e-5
    b = pr["b"]
    for i in range(b.shape[0]):
        if pr["parent"][i] < 0:
            continue
        bp, bm = b.copy(), b.copy()
        bp[i] += h
        bm[i] -= h
        fd = (oracle_mod.evaluate(pr, bp).grad[i] - oracle_mod.evaluate(pr, bm).grad[i]) / (2 * h)
        assert abs(fd - r.hess[i]) <= 1e-5 * max(1.0, abs(r.hess[i]))


def test_indicator_and_all_ones_rows_are_the_plain_codes(oracle_mod):
    m = 4
    pr = wl.random_problem(12, 80, n_states=m, n_cat=2, seed=41, b_mean=0.2, ambiguous=0.1)
    plain = oracle_mod.evaluate(pr)
    table = np.vstack([np.eye(m), np.ones((1, m))])   # codes m..m+3: states, m+4: all ones
    tips = pr["tip_states"].copy()
    tips = np.where(tips < m, tips + m, m + 4).astype(np.uint8)
    r = oracle_mod.evaluate(dict(pr, tip_partials=table, tip_states=tips))
    assert r.logL == plain.logL
    np.testing.assert_array_equal(r.grad, plain.grad)
    np.testing.assert_array_equal(r.hess, plain.hess)
    # codes past the table are missing data
    tips2 = np.where(pr["tip_states"] < m, pr["tip_states"], wl.MISSING).astype(np.uint8)
    r2 = oracle_mod.evaluate(dict(pr, tip_partials=table, tip_states=tips2))
    assert r2.logL == plain.logL


@pytest.mark.parametrize("bad", ["negative", "zero", "nan", "shape"])
def test_rejects_invalid_tip_vectors(oracle_mod, bad):
    pr = wl.random_problem(5, 10, n_states=4, seed=51)
    table = wl.iupac_nucleotide_partials()
    if bad == "negative":
        table[2, 1] = -0.1
    elif bad == "zero":
        table[3] = 0.0
    elif bad == "nan":
        table[0, 0] = np.nan
    else:
        table = table[:, :3]
    with pytest.raises(ValueError):
        oracle_mod.evaluate(dict(pr, tip_partials=table))


def test_per_cell_partials_encode_to_codes_and_a_table(oracle_mod):
    """Per-cell vectors [N][P][m] (one partial vector for every tip and pattern) reduce to codes and a
    table that reproduce every cell; the oracle gives the same result on both encodings of a
    problem whose per-cell form was built from codes."""
    m = 4
    pr = _partial_problem(9, 70, 91)
    V = ind.tip_vectors(pr, m)
    cells = V[pr["tip_states"]]                       # [N][P][m]
    codes, table = wl.encode_tip_partials(cells)
    np.testing.assert_array_equal(ind.tip_vectors(dict(tip_partials=table), m)[codes], cells)
    assert table.shape[0] <= len(pr["tip_partials"])
    r0 = oracle_mod.evaluate(pr)
    r1 = oracle_mod.evaluate(dict(pr, tip_states=codes, tip_partials=table))
    assert abs(r1.logL - r0.logL) <= 1e-13 * abs(r0.logL)
    np.testing.assert_allclose(r1.grad, r0.grad, rtol=1e-12, atol=1e-14)
    with pytest.raises(ValueError):   # too many distinct vectors for one-byte codes
        wl.encode_tip_partials(np.random.default_rng(0).random((2, 300, m)))
