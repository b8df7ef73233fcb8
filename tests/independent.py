"""Independent computations that pin the oracle (and through it the CUDA path).

Nothing here is shared with ``oracle/`` or with the library.  Transition matrices come from
``scipy.linalg.expm`` (the oracle uses its own Pade code).  The likelihood is computed from its
definition as a sum over every assignment of internal states (Eq. 1 with the rate mixture of
Section 2.5), the gradient either by differentiating that sum term by term or by the quadratic
"substitute dP for P and prune again" scheme the paper compares against (Section 1).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla


def _model(problem, i):
    bm = problem.get("branch_model")
    return 0 if bm is None else int(bm[i])


def tip_vectors(problem, m):
    """V[256][m]: the tip partial vector of every code (Section 2.1): the indicator of state y for
    y < m, row y - m of problem["tip_partials"] for the next K codes, all ones after them."""
    V = np.ones((256, m))
    V[:m] = np.eye(m)
    tv = problem.get("tip_partials")
    if tv is not None and len(tv):
        V[m:m + len(tv)] = tv
    return V


def transition_matrices(problem, b):
    """P[i][l] = expm(Q_i b_i r_l) and dP[i][l] = r_l Q_i P[i][l] (d/db_i) via scipy."""
    n = problem["parent"].shape[0]
    Q = problem["Q"]
    rates = problem["cat_rates"]
    P, dP = {}, {}
    for i in range(n):
        if problem["parent"][i] < 0:
            continue
        Qi = Q[_model(problem, i)]
        for l, r in enumerate(rates):
            Pm = sla.expm(Qi * b[i] * r)
            P[i, l] = Pm
            dP[i, l] = r * Qi @ Pm
    return P, dP


def brute_force(problem, b=None):
    """Eq. 1 summed over all m^(N-1) internal-state assignments, for every site pattern.

    Returns (site likelihoods L[P], d L / d b_i [n][P]).  The derivative of each product term
    with respect to b_i replaces the factor P_i[y_pa, y_i] by dP_i[y_pa, y_i]."""
    b = problem["b"] if b is None else b
    parent = problem["parent"]
    n = parent.shape[0]
    N = int(problem.get("n_tips", (n + 1) // 2))
    m = problem["Q"].shape[1]
    tips = problem["tip_states"].astype(np.int64)
    n_pat = tips.shape[1]
    pi = problem["root_freqs"]
    cw = problem["cat_weights"]
    P, dP = transition_matrices(problem, b)
    root = int(np.flatnonzero(parent < 0)[0])
    internal = list(range(N, n))
    L = np.zeros(n_pat)
    dL = np.zeros((n, n_pat))
    branches = [i for i in range(n) if i != root]
    V = tip_vectors(problem, m)
    for assign in itertools.product(range(m), repeat=len(internal)):
        y = dict(zip(internal, assign))
        for l in range(len(cw)):
            factors = {}
            dfactors = {}
            for i in branches:
                a = y[int(parent[i])]
                if i < N:   # sum over the tip's state, weighted by its partial vector
                    factors[i] = V[tips[i]] @ P[i, l][a]
                    dfactors[i] = V[tips[i]] @ dP[i, l][a]
                else:
                    factors[i] = np.full(n_pat, P[i, l][a, y[i]])
                    dfactors[i] = np.full(n_pat, dP[i, l][a, y[i]])
            base = cw[l] * pi[y[root]]
            term = np.full(n_pat, base)
            for i in branches:
                term = term * factors[i]
            L += term
            for j in branches:
                d = np.full(n_pat, base)
                for i in branches:
                    d = d * (dfactors[i] if i == j else factors[i])
                dL[j] += d
    return L, dL


def prune(problem, P, replace=None):
    """Plain recursive pruning (no scaling) with optionally one branch's matrices replaced.

    ``replace`` = (branch, {l: matrix}).  Returns the site likelihoods."""
    parent = problem["parent"]
    n = parent.shape[0]
    N = int(problem.get("n_tips", (n + 1) // 2))
    m = problem["Q"].shape[1]
    C = len(problem["cat_weights"])
    tips = problem["tip_states"]
    n_pat = tips.shape[1]
    kids = [[] for _ in range(n)]
    for i, p in enumerate(parent):
        if p >= 0:
            kids[int(p)].append(i)
    root = int(np.flatnonzero(parent < 0)[0])

    def mat(i, l):
        if replace is not None and replace[0] == i:
            return replace[1][l]
        return P[i, l]

    V = tip_vectors(problem, m)

    def vec(k):  # [C][m][P]
        if k < N:
            return np.repeat(V[tips[k]].T[None], C, axis=0)
        out = np.ones((C, m, n_pat))
        for c in kids[k]:
            vc = vec(c)
            for l in range(C):
                out[l] *= mat(c, l) @ vc[l]
        return out

    vr = vec(root)
    pi = problem["root_freqs"]
    cw = problem["cat_weights"]
    return sum(cw[l] * (pi @ vr[l]) for l in range(C))


def quadratic_gradient(problem, b=None):
    """O(N^2) gradient: for each branch, prune again with dP_i in place of P_i (Section 1)."""
    b = problem["b"] if b is None else b
    P, dP = transition_matrices(problem, b)
    n = problem["parent"].shape[0]
    C = len(problem["cat_weights"])
    L = prune(problem, P)
    w = problem["weights"]
    g = np.zeros(n)
    for i in range(n):
        if problem["parent"][i] < 0:
            continue
        dL = prune(problem, P, replace=(i, {l: dP[i, l] for l in range(C)}))
        g[i] = float(np.sum(w * dL / L))
    return g, float(np.sum(w * np.log(L)))


def reroot(parent, b, edge_child, frac):
    """Move the root of a binary tree onto the edge above ``edge_child`` at fraction ``frac``
    of its length (measured from the child).  The old root's two edges merge into one.  Node
    labels are kept (the old root's label becomes the new root).  Returns (parent, b)."""
    n = parent.shape[0]
    root = int(np.flatnonzero(parent < 0)[0])
    kids = [int(i) for i in np.flatnonzero(parent == root)]
    adj = {i: {} for i in range(n) if i != root}
    for i in range(n):
        p = int(parent[i])
        if p < 0 or p == root:
            continue
        adj[i][p] = b[i]
        adj[p][i] = b[i]
    a, c = kids
    adj[a][c] = b[a] + b[c]
    adj[c][a] = b[a] + b[c]
    x = edge_child
    y = int(parent[x]) if int(parent[x]) != root else (c if x == a else a)
    length = adj[x][y]
    del adj[x][y]
    del adj[y][x]
    new_parent = np.full(n, -1, dtype=np.int32)
    new_b = np.zeros(n)
    new_parent[x] = root
    new_parent[y] = root
    new_b[x] = frac * length
    new_b[y] = (1.0 - frac) * length
    stack = [x, y]
    while stack:
        u = stack.pop()
        for v, lv in adj[u].items():
            if v == int(new_parent[u]) or new_parent[v] != -1 or v in (x, y):
                continue
            new_parent[v] = u
            new_b[v] = lv
            stack.append(v)
    return new_parent, new_b


def resolve_zero_length(problem):
    """A tree with multifurcations as a binary tree: a node with d > 2 children keeps its last child
    and an added node, which keeps the next-to-last child and another added node, and so on; the
    last added node takes the first two children.  The d - 2 added branches have length 0 (their
    transition matrices are the identity).  The original nodes keep their ids; the added ones come
    after them.  Returns the binary problem (b included) and the number of original nodes."""
    parent = np.asarray(problem["parent"], dtype=np.int64)
    n = parent.shape[0]
    N = int(problem["n_tips"])
    kids = [[] for _ in range(n)]
    for i, p in enumerate(parent):
        if p >= 0:
            kids[int(p)].append(i)
    new_parent = list(int(p) for p in parent)
    b = list(problem["b"])
    for k in range(n):
        ch = kids[k]
        if len(ch) <= 2:
            continue
        at = k
        for j in range(len(ch) - 1, 1, -1):
            new_parent[ch[j]] = at
            x = len(new_parent)
            new_parent.append(at)
            b.append(0.0)
            at = x
        new_parent[ch[0]] = at
        new_parent[ch[1]] = at
    assert len(new_parent) == 2 * N - 1
    out = dict(problem, parent=np.array(new_parent, dtype=np.int32), b=np.array(b), n_tips=N)
    bm = problem.get("branch_model")
    if bm is not None:
        out["branch_model"] = np.concatenate([np.asarray(bm, dtype=np.int32),
                                              np.zeros(len(new_parent) - n, dtype=np.int32)])
    return out, n
