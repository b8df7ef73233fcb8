"""Writes the stored expected values under tests/golden/ by calling only the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle  # noqa: E402


def fig1_three_taxon():
    """The 3-taxon tree of Fig. 1 / Eq. (pruningVec), 0-based: tips 0,1,2 (paper 1,2,3),
    node 3 = parent of tips 0 and 1 (paper 4), root 4 = parent of 3 and tip 2 (paper 5).
    JC69 generator, uniform root frequencies, one rate category, five site patterns (the last
    one has tip 2 missing)."""
    q = np.full((4, 4), 1.0 / 3.0)
    np.fill_diagonal(q, -1.0)
    inputs = {
        "citation": "Fig. 1 and Eq. (pruningVec), Section 2.3; Eq. (preOrderUpdate), Section 2.4",
        "parent": [3, 3, 4, 4, -1],
        "tip_states": [[0, 0, 1, 3, 2], [0, 2, 1, 0, 2], [0, 0, 3, 1, 4]],
        "weights": [3.0, 1.0, 2.0, 1.0, 1.0],
        "Q": q.tolist(),
        "root_freqs": [0.25, 0.25, 0.25, 0.25],
        "cat_rates": [1.0],
        "cat_weights": [1.0],
        "b": [0.11, 0.23, 0.37, 0.05, 0.0],
    }
    pr = {k: np.asarray(v) for k, v in inputs.items() if k != "citation"}
    pr["parent"] = pr["parent"].astype(np.int32)
    pr["tip_states"] = pr["tip_states"].astype(np.uint8)
    pr["Q"] = pr["Q"][None]
    r = oracle.evaluate(pr)
    inputs["expected"] = {"logL": r.logL, "grad": r.grad.tolist(),
                          "site_logL": r.site_logL.tolist(), "hess": r.hess.tolist()}
    return inputs


if __name__ == "__main__":
    with open(os.path.join(HERE, "fig1_three_taxon.json"), "w") as f:
        json.dump(fig1_three_taxon(), f, indent=1)
        f.write("\n")
