"""The paper's worked example (Fig. 1): stored oracle values, and the same numbers from the
paper's explicit forms for that tree with closed-form JC69 transition matrices (no expm)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _load():
    with open(os.path.join(HERE, "golden", "fig1_three_taxon.json")) as f:
        return json.load(f)


def _problem(g):
    pr = {k: np.asarray(v) for k, v in g.items() if k not in ("citation", "expected")}
    pr["parent"] = pr["parent"].astype(np.int32)
    pr["tip_states"] = pr["tip_states"].astype(np.uint8)
    pr["Q"] = pr["Q"][None]
    return pr


def _jc(t):
    e = np.exp(-4.0 * t / 3.0)
    P = np.full((4, 4), 0.25 - 0.25 * e)
    np.fill_diagonal(P, 0.25 + 0.75 * e)
    return P


def test_oracle_reproduces_stored_values(oracle_mod):
    g = _load()
    r = oracle_mod.evaluate(_problem(g))
    exp = g["expected"]
    assert abs(r.logL - exp["logL"]) <= 1e-13 * abs(exp["logL"])
    np.testing.assert_allclose(r.grad, exp["grad"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(r.site_logL, exp["site_logL"], rtol=1e-13)
    np.testing.assert_allclose(r.hess, exp["hess"], rtol=1e-12, atol=1e-14)


def test_stored_values_match_worked_example_closed_form():
    """Eq. (pruningVec): P(Y) = pi' [P4 (P1 p1 o P2 p2) o P3 p3]; the gradient on branch 4 from
    the example q4 = P4' [q5 o (P3 p3)] with q5 = pi and Eq. (singleRateCaseGradient)."""
    g = _load()
    b = np.asarray(g["b"])
    Q = np.asarray(g["Q"])
    pi = np.asarray(g["root_freqs"])
    w = np.asarray(g["weights"])
    tips = np.asarray(g["tip_states"])
    P1, P2, P3, P4 = _jc(b[0]), _jc(b[1]), _jc(b[2]), _jc(b[3])
    logL, grad4 = 0.0, 0.0
    site = []
    for s in range(tips.shape[1]):
        p1, p2, p3 = (np.ones(4) if tips[t, s] >= 4 else np.eye(4)[tips[t, s]] for t in range(3))
        p4 = (P1 @ p1) * (P2 @ p2)
        L = pi @ ((P4 @ p4) * (P3 @ p3))
        q4 = P4.T @ (pi * (P3 @ p3))
        site.append(np.log(L))
        logL += w[s] * np.log(L)
        grad4 += w[s] * (q4 @ Q @ p4) / L
    exp = g["expected"]
    np.testing.assert_allclose(exp["site_logL"], site, rtol=1e-14)
    assert abs(exp["logL"] - logL) <= 1e-14 * abs(logL)
    assert abs(exp["grad"][3] - grad4) <= 1e-12 * abs(grad4)
