"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module generates INPUTS only: trees, branch lengths, substitution generators Q, root
frequencies, discrete rate categories and alignments. It contains none of the method's
arithmetic (no matrix exponential, no pruning, no pre-order pass, no gradient): sites are
simulated down the tree with an exact jump-chain (Gillespie) simulation of the CTMC, which needs
only the entries of Q, never e^{Qt}.

Conventions (Section 2.1 of the paper, 0-based): tips are nodes 0..N-1, internal nodes N..2N-2,
the root is the node whose parent is -1.  A branch is named by its child node.  A problem is a
plain dict of numpy arrays; every generator takes an explicit ``numpy.random.Generator``.
"""
from __future__ import annotations

import numpy as np
from scipy import special, stats

# --------------------------------------------------------------------------------------------
# trees
# --------------------------------------------------------------------------------------------


def yule_tree(n_tips: int, rng: np.random.Generator, birth_rate: float = 1.0):
    """Random rooted binary tree from a pure-birth (Yule) process.

    Returns ``(parent, node_time)``.  ``parent`` is int32[2N-1] with tips 0..N-1, internal
    N..2N-2 and the root 2N-2 (parent -1); every internal node has a larger index than its
    children, as in the paper's numbering.  ``node_time`` is the forward time of each node
    (root at 0, tips at the time the process reached N lineages).
    """
    if n_tips < 2:
        raise ValueError("a tree needs at least two tips")
    n_nodes = 2 * n_tips - 1
    # Grow top-down: lineages are open branches whose lower node is not yet decided.
    # Internal nodes are labelled in creation order and relabelled at the end so that the
    # root is 2N-2 and labels decrease towards the tips.
    created_parent = [-1]          # parent (creation label) of internal node in creation order
    created_time = [0.0]
    t = 0.0
    lineage_parent = [0, 0]
    while len(lineage_parent) < n_tips:
        k = len(lineage_parent)
        t += rng.exponential(1.0 / (birth_rate * k))
        pick = int(rng.integers(k))
        par = lineage_parent.pop(pick)
        label = len(created_parent)
        created_parent.append(par)
        created_time.append(t)
        lineage_parent.extend([label, label])
    t_end = t + rng.exponential(1.0 / (birth_rate * n_tips))
    n_int = len(created_parent)
    assert n_int == n_tips - 1
    # relabel: creation label c -> node id 2N-2-c
    parent = np.full(n_nodes, -1, dtype=np.int32)
    node_time = np.zeros(n_nodes, dtype=np.float64)
    for c in range(n_int):
        node = 2 * n_tips - 2 - c
        parent[node] = -1 if created_parent[c] < 0 else 2 * n_tips - 2 - created_parent[c]
        node_time[node] = created_time[c]
    order = rng.permutation(n_tips)  # tips get labels in random order
    for j, par in enumerate(lineage_parent):
        tip = int(order[j])
        parent[tip] = 2 * n_tips - 2 - par
        node_time[tip] = t_end
    return parent, node_time


def caterpillar_tree(n_tips: int):
    """Fully unbalanced (ladder) tree: height N-1, the worst case for level scheduling."""
    n_nodes = 2 * n_tips - 1
    parent = np.full(n_nodes, -1, dtype=np.int32)
    # internal node N + i joins internal node N + i - 1 (or tip 0) with tip i + 1
    for i in range(n_tips - 1):
        node = n_tips + i
        left = 0 if i == 0 else n_tips + i - 1
        parent[left] = node
        parent[i + 1] = node
    return parent


def relabel_nodes(parent: np.ndarray, rng: np.random.Generator, n_tips: int):
    """Random relabelling of internal nodes (tips keep 0..N-1): the library must not rely on
    any particular internal numbering.  Returns ``(new_parent, perm)`` with new id = perm[old]."""
    n_nodes = parent.shape[0]
    perm = np.arange(n_nodes)
    perm[n_tips:] = n_tips + rng.permutation(n_nodes - n_tips)
    new_parent = np.full(n_nodes, -1, dtype=np.int32)
    for old in range(n_nodes):
        if parent[old] >= 0:
            new_parent[perm[old]] = perm[parent[old]]
    return new_parent, perm


def children_lists(parent: np.ndarray):
    kids = [[] for _ in range(parent.shape[0])]
    for i, p in enumerate(parent):
        if p >= 0:
            kids[int(p)].append(i)
    return kids


def root_of(parent: np.ndarray) -> int:
    roots = np.flatnonzero(parent < 0)
    assert roots.size == 1
    return int(roots[0])


def collapse_edges(parent: np.ndarray, n_tips: int, nodes, b: np.ndarray | None = None):
    """A tree with multifurcations: every internal non-root node in ``nodes`` is removed and its
    children are attached to its parent (its branch disappears).  The remaining internal nodes are
    renumbered in order to stay contiguous after the tips.  Returns ``(parent, b, old)`` with
    ``old[new_id]`` the node's id in the input tree (``b`` follows the kept nodes; None if not given)."""
    parent = np.asarray(parent, dtype=np.int64)
    n = parent.shape[0]
    drop = set(int(x) for x in nodes)
    for x in drop:
        if x < n_tips or parent[x] < 0:
            raise ValueError(f"node {x} is a tip or the root")
    keep = [i for i in range(n) if i not in drop]
    new_id = {old: new for new, old in enumerate(keep)}

    def kept_ancestor(i):
        p = int(parent[i])
        while p in drop:
            p = int(parent[p])
        return p

    out = np.full(len(keep), -1, dtype=np.int32)
    for new, old in enumerate(keep):
        if parent[old] >= 0:
            out[new] = new_id[kept_ancestor(old)]
    old_arr = np.array(keep, dtype=np.int64)
    return out, (None if b is None else np.asarray(b, dtype=np.float64)[old_arr]), old_arr


def multifurcating_problem(n_tips, n_patterns, n_collapse, n_states=4, n_cat=1, seed=0, **kw):
    """random_problem on a Yule tree, then ``n_collapse`` random internal branches collapsed
    (collapse_edges): nodes of degree 3 and more, the data simulated on the binary tree."""
    pr = random_problem(n_tips, n_patterns, n_states=n_states, n_cat=n_cat, seed=seed, **kw)
    rng = np.random.default_rng(seed + 1000)
    root = root_of(pr["parent"])
    cand = [i for i in range(n_tips, pr["parent"].shape[0]) if i != root]
    nodes = rng.choice(cand, size=min(n_collapse, len(cand)), replace=False)
    parent, b, old = collapse_edges(pr["parent"], n_tips, nodes, pr["b"])
    out = dict(pr, parent=parent, b=b, n_tips=n_tips)
    if pr.get("branch_model") is not None:
        out["branch_model"] = np.ascontiguousarray(pr["branch_model"][old], dtype=np.int32)
    out["node_time"] = None
    return out


def branch_lengths(parent: np.ndarray, mean: float, rng: np.random.Generator):
    """b_i ~ Exp(mean) for every non-root node; the root entry is 0."""
    b = rng.exponential(mean, size=parent.shape[0])
    b[parent < 0] = 0.0
    return b


# --------------------------------------------------------------------------------------------
# substitution models
# --------------------------------------------------------------------------------------------


def stationary_distribution(Q: np.ndarray) -> np.ndarray:
    """Left null vector of Q normalised to sum 1 (input normalisation only)."""
    m = Q.shape[0]
    A = np.vstack([Q.T, np.ones((1, m))])
    rhs = np.zeros(m + 1)
    rhs[-1] = 1.0
    pi, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    return pi


def normalise_rate(Q: np.ndarray) -> np.ndarray:
    """Scale Q so that the expected substitution rate at stationarity is 1."""
    pi = stationary_distribution(Q)
    rate = -float(np.dot(pi, np.diag(Q)))
    return Q / rate


def random_general_Q(m: int, rng: np.random.Generator, lo: float = 0.1, hi: float = 1.0,
                     normalise: bool = True) -> np.ndarray:
    """General non-reversible generator: off-diagonals U(lo, hi), rows sum to zero."""
    Q = rng.uniform(lo, hi, size=(m, m))
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    return normalise_rate(Q) if normalise else Q


def random_reversible_Q(m: int, rng: np.random.Generator, pi: np.ndarray | None = None):
    """GTR-style reversible generator Q_ij = s_ij pi_j with symmetric exchangeabilities."""
    if pi is None:
        pi = rng.dirichlet(np.ones(m))
    S = rng.uniform(0.1, 1.0, size=(m, m))
    S = np.triu(S, 1)
    S = S + S.T
    Q = S * pi[None, :]
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    return normalise_rate(Q), pi


def jc69_Q() -> np.ndarray:
    Q = np.full((4, 4), 1.0 / 3.0)
    np.fill_diagonal(Q, -1.0)
    return Q


def dirichlet_freqs(m: int, rng: np.random.Generator) -> np.ndarray:
    return rng.dirichlet(np.ones(m))


def discrete_gamma(shape: float, n_cat: int):
    """Yang (1994) discrete gamma, mean of each equal-probability category; mean rate 1.

    Returns ``(rates, weights)``.  The paper cites this scheme for rate heterogeneity but fixes
    no discretisation, so the library takes rates and weights as inputs."""
    if n_cat == 1:
        return np.ones(1), np.ones(1)
    cuts = stats.gamma.ppf(np.arange(1, n_cat) / n_cat, a=shape, scale=1.0 / shape)
    edges = np.concatenate([[0.0], cuts, [np.inf]])
    upper = special.gammainc(shape + 1.0, edges * shape)
    rates = n_cat * np.diff(upper)
    return rates, np.full(n_cat, 1.0 / n_cat)


# standard genetic code, codons in TCAG order for positions 1, 2, 3
_BASES = "TCAG"
_AA = "FFLLSSSSYY**CC*WLLLLPPPPHHQQRRRRIIIMTTTTNNKKSSRRVVVVAAAADDEEGGGG"


def sense_codons():
    """The 61 sense codons of the standard code as (codon string, amino acid)."""
    out = []
    for i, a in enumerate(_BASES):
        for j, b in enumerate(_BASES):
            for k, c in enumerate(_BASES):
                aa = _AA[16 * i + 4 * j + k]
                if aa != "*":
                    out.append((a + b + c, aa))
    return out


def codon_Q(rng: np.random.Generator, omega: float = 0.3, pi: np.ndarray | None = None):
    """Reversible codon generator (61 states): single-nucleotide changes only, rate =
    exchangeability(nucleotide pair; 6 values U(0.1,1)) * pi_target * (omega if the change is
    nonsynonymous).  Returns ``(Q, pi)`` with Q normalised to rate 1."""
    codons = sense_codons()
    m = len(codons)
    if pi is None:
        pi = rng.dirichlet(np.ones(m))
    pairs = {}
    vals = rng.uniform(0.1, 1.0, size=6)
    idx = 0
    for x in range(4):
        for y in range(x + 1, 4):
            pairs[(x, y)] = pairs[(y, x)] = vals[idx]
            idx += 1
    Q = np.zeros((m, m))
    for a, (ca, aa_a) in enumerate(codons):
        for b, (cb, aa_b) in enumerate(codons):
            diff = [p for p in range(3) if ca[p] != cb[p]]
            if len(diff) != 1:
                continue
            p = diff[0]
            s = pairs[(_BASES.index(ca[p]), _BASES.index(cb[p]))]
            Q[a, b] = s * pi[b] * (1.0 if aa_a == aa_b else omega)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    return normalise_rate(Q), pi


# --------------------------------------------------------------------------------------------
# alignments
# --------------------------------------------------------------------------------------------


def _jump_chain(states, lengths, Q, rng):
    """Exact CTMC simulation along independent branches of the given lengths (one per site)."""
    m = Q.shape[0]
    out_rate = -np.diag(Q)
    jump = Q.copy()
    np.fill_diagonal(jump, 0.0)
    jump_cdf = np.cumsum(jump / out_rate[:, None], axis=1)
    jump_cdf[:, -1] = 1.0
    s = states.copy()
    remaining = lengths.copy()
    active = np.flatnonzero(remaining > 0)
    while active.size:
        wait = rng.exponential(1.0 / out_rate[s[active]])
        jumped = wait < remaining[active]
        remaining[active] -= wait
        idx = active[jumped]
        if idx.size:
            u = rng.random(idx.size)
            s[idx] = (jump_cdf[s[idx]] < u[:, None]).sum(axis=1)
            np.minimum(s, m - 1, out=s)
        active = idx
    return s


def simulate_alignment(parent, b, Q, pi, cat_rates, cat_weights, n_sites, rng,
                       branch_model=None):
    """Simulate ``n_sites`` columns down the tree: root state ~ pi, a rate category per site,
    jump-chain evolution along each branch for time b_i * rate.  Returns uint8[N][n_sites]."""
    n_nodes = parent.shape[0]
    n_tips = (n_nodes + 1) // 2
    Qs = Q if Q.ndim == 3 else Q[None]
    kids = children_lists(parent)
    root = root_of(parent)
    cat = rng.choice(len(cat_rates), size=n_sites, p=cat_weights)
    site_rate = np.asarray(cat_rates)[cat]
    state = {root: rng.choice(len(pi), size=n_sites, p=pi)}
    stack = [root]
    while stack:
        k = stack.pop()
        for c in kids[k]:
            model = 0 if branch_model is None else int(branch_model[c])
            state[c] = _jump_chain(state[k], b[c] * site_rate, Qs[model], rng)
            stack.append(c)
    return np.stack([state[t] for t in range(n_tips)]).astype(np.uint8)


def make_ambiguous(tips: np.ndarray, frac: float, n_states: int, rng):
    """Set a fraction of tip cells to the all-ones (missing / fully ambiguous) code n_states."""
    out = tips.copy()
    mask = rng.random(out.shape) < frac
    out[mask] = n_states
    return out


MISSING = 255   # a tip code past every row of a tip-partial table: missing data (all ones)


def iupac_nucleotide_partials(error: float = 0.0) -> np.ndarray:
    """Partial vectors of the ten IUPAC ambiguity codes that name 2 or 3 of the states (A, C, G,
    T) = (0, 1, 2, 3): R, Y, S, W, K, M, B, D, H, V as 0/1 vectors.  With ``error`` > 0, four rows
    follow for a base call with that error probability spread over the other three states."""
    sets = ["AG", "CT", "CG", "AT", "GT", "AC", "CGT", "AGT", "ACT", "ACG"]
    rows = [[1.0 if c in s else 0.0 for c in "ACGT"] for s in sets]
    if error > 0:
        rows += [[1.0 - error if j == y else error / 3 for j in range(4)] for y in range(4)]
    return np.array(rows)


def make_partially_observed(tips: np.ndarray, frac: float, table: np.ndarray, rng):
    """Recode a fraction of the observed cells (code < m) as partial observations: code m + k
    for a row k of ``table`` [K][m] drawn among the rows that allow the cell's state.  Cells that
    were missing (code >= m) become ``MISSING``, past the table's codes."""
    K, m = table.shape
    if m + K > MISSING:
        raise ValueError("the table leaves no code for missing data")
    out = tips.copy()
    out[tips >= m] = MISSING
    allow = [np.flatnonzero(table[:, y] > 0) for y in range(m)]
    for idx in zip(*np.nonzero((tips < m) & (rng.random(tips.shape) < frac))):
        rows = allow[tips[idx]]
        if rows.size:
            out[idx] = m + rows[rng.integers(rows.size)]
    return out


def encode_tip_partials(partials: np.ndarray):
    """Per-cell tip partial vectors [N][P][m] as (codes [N][P] uint8, table [K][m]): an indicator
    vector becomes its state, an all-ones vector the missing code, every other distinct vector a
    row of the table (code m + row).  Raises ValueError when more than 255 - m distinct vectors
    remain."""
    partials = np.asarray(partials, dtype=np.float64)
    N, P, m = partials.shape
    flat = partials.reshape(-1, m)
    codes = np.full(flat.shape[0], MISSING, dtype=np.uint8)
    ones = np.all(flat == 1.0, axis=1)
    onehot = (np.sum(flat == 1.0, axis=1) == 1) & (np.sum(flat == 0.0, axis=1) == m - 1)
    codes[onehot] = np.argmax(flat[onehot], axis=1)
    rest = ~(ones | onehot)
    table, inverse = np.unique(flat[rest], axis=0, return_inverse=True)
    if m + table.shape[0] > MISSING:
        raise ValueError(f"{table.shape[0]} distinct partial vectors leave no code for missing data")
    codes[rest] = m + inverse.reshape(-1)
    return codes.reshape(N, P), table


# --------------------------------------------------------------------------------------------
# problems
# --------------------------------------------------------------------------------------------


def make_problem(parent, tip_states, weights, Q, pi, cat_rates, cat_weights, b,
                 branch_model=None, node_time=None):
    n_nodes = parent.shape[0]
    Qs = np.ascontiguousarray(Q if Q.ndim == 3 else Q[None], dtype=np.float64)
    return {
        "parent": np.ascontiguousarray(parent, dtype=np.int32),
        "tip_states": np.ascontiguousarray(tip_states, dtype=np.uint8),
        "weights": np.ascontiguousarray(weights, dtype=np.float64),
        "Q": Qs,
        "branch_model": None if branch_model is None else np.ascontiguousarray(branch_model, dtype=np.int32),
        "root_freqs": np.ascontiguousarray(pi, dtype=np.float64),
        "cat_rates": np.ascontiguousarray(cat_rates, dtype=np.float64),
        "cat_weights": np.ascontiguousarray(cat_weights, dtype=np.float64),
        "b": np.ascontiguousarray(b, dtype=np.float64),
        "n_tips": (n_nodes + 1) // 2,
        "n_states": Qs.shape[1],
        "node_time": node_time,
    }


def random_problem(n_tips, n_patterns, n_states=4, n_cat=1, seed=0, b_mean=0.05,
                   ambiguous=0.0, gamma_shape=0.5, reversible=False, tree="yule",
                   weights="unit", n_models=1, relabel=False):
    """General-purpose seeded problem used by tests (any state count, tree shape, categories)."""
    rng = np.random.default_rng(seed)
    if tree == "yule":
        parent, node_time = yule_tree(n_tips, rng)
    elif tree == "caterpillar":
        parent, node_time = caterpillar_tree(n_tips), None
    else:
        raise ValueError(tree)
    if relabel:
        parent, _ = relabel_nodes(parent, rng, n_tips)
    b = branch_lengths(parent, b_mean, rng)
    if n_states == 61:
        Q0, pi = codon_Q(rng)
        Qs = [Q0] + [codon_Q(rng, pi=pi)[0] for _ in range(n_models - 1)]
    elif reversible:
        Q0, pi = random_reversible_Q(n_states, rng)
        Qs = [Q0] + [random_reversible_Q(n_states, rng, pi)[0] for _ in range(n_models - 1)]
    else:
        Qs = [random_general_Q(n_states, rng) for _ in range(n_models)]
        pi = dirichlet_freqs(n_states, rng)
    Q = np.stack(Qs)
    branch_model = None
    if n_models > 1:
        branch_model = rng.integers(0, n_models, size=parent.shape[0]).astype(np.int32)
    rates, cw = discrete_gamma(gamma_shape, n_cat)
    tips = simulate_alignment(parent, b, Q, pi, rates, cw, n_patterns, rng, branch_model)
    if ambiguous > 0:
        tips = make_ambiguous(tips, ambiguous, n_states, rng)
    if weights == "unit":
        w = np.ones(n_patterns)
    elif weights == "int":
        w = rng.integers(1, 6, size=n_patterns).astype(np.float64)
    else:
        raise ValueError(weights)
    return make_problem(parent, tips, w, Q, pi, rates, cw, b, branch_model, node_time)


def config_small(seed: int = 0):
    """16-taxon Yule tree, b ~ Exp(0.05), general non-reversible 4x4 Q (off-diagonals U(0.1,1)),
    Dirichlet root frequencies, 500 patterns with integer weights 1..5, one rate category."""
    return random_problem(16, 500, n_states=4, n_cat=1, seed=seed, b_mean=0.05, weights="int")


def config_nucleotide(seed: int = 1, n_tips: int = 1000, n_patterns: int = 10000):
    """1,000-taxon Yule tree, b ~ Exp(0.01), non-reversible 4x4 Q, 4 discrete-gamma categories
    (shape 0.5), 10,000 simulated patterns (weight 1) with 2% all-ones ambiguous tip cells."""
    return random_problem(n_tips, n_patterns, n_states=4, n_cat=4, seed=seed, b_mean=0.01,
                          ambiguous=0.02, gamma_shape=0.5)


def config_codon(seed: int = 2, n_tips: int = 500, n_patterns: int = 3000):
    """500-taxon Yule tree, b ~ Exp(0.01), reversible codon Q (omega 0.3, random codon
    frequencies), 3,000 simulated codon patterns, 4 discrete-gamma categories (shape 0.5)."""
    return random_problem(n_tips, n_patterns, n_states=61, n_cat=4, seed=seed, b_mean=0.01,
                          gamma_shape=0.5)


def config_clock_batch(seed: int = 3, n_trees: int = 64, n_tips: int = 300,
                       n_patterns: int = 5000, b_mean_target: float = 0.01):
    """Independent Yule trees with a random-effects clock: b_i = mu * eps_i * (t_i - t_pa(i)),
    eps_i ~ lognormal(0, 0.5); mu chosen so the mean branch length is about ``b_mean_target``.
    One rate category, 5,000 nucleotide patterns each.  Returns a list of problems, each with
    extra keys ``dt`` (branch durations), ``eps`` and ``mu``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_trees):
        parent, node_time = yule_tree(n_tips, rng)
        dt = np.zeros(parent.shape[0])
        nz = parent >= 0
        dt[nz] = node_time[nz] - node_time[parent[nz]]
        eps = rng.lognormal(0.0, 0.5, size=parent.shape[0])
        mu = b_mean_target / float(np.mean(dt[nz] * eps[nz]))
        b = mu * eps * dt
        Q = random_general_Q(4, rng)
        pi = dirichlet_freqs(4, rng)
        tips = simulate_alignment(parent, b, Q, pi, np.ones(1), np.ones(1), n_patterns, rng)
        pr = make_problem(parent, tips, np.ones(n_patterns), Q, pi, np.ones(1), np.ones(1), b,
                          node_time=node_time)
        pr.update(dt=dt, eps=eps, mu=mu)
        out.append(pr)
    return out


def serving_requests(n_requests: int, seed: int = 5, taxa=(50, 2000), patterns=(500, 20000),
                     p_codon=0.2, max_cat=4):
    """Request descriptors for the serving stream: taxa U{50..2000}, patterns U{500..20000},
    4 states with probability 0.8 else 61, 1..4 rate categories.  Only shapes and seeds are
    drawn here; ``materialise_request`` builds the arrays."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_requests):
        reqs.append({
            "id": i,
            "n_tips": int(rng.integers(taxa[0], taxa[1] + 1)),
            "n_patterns": int(rng.integers(patterns[0], patterns[1] + 1)),
            "n_states": 61 if rng.random() < p_codon else 4,
            "n_cat": int(rng.integers(1, max_cat + 1)),
            "seed": int(rng.integers(2**31)),
        })
    return reqs


def serving_masters(max_taxa: int = 2000, max_patterns: int = 20000, seed: int = 6, ambiguous: float = 0.02):
    """Seeded tip-state matrices [max_taxa, max_patterns] for 4 and 61 states (i.i.d. codes, a
    fraction ``ambiguous`` set to the all-ones code).  A serving request takes a row-strided view
    of its taxa x patterns block, so generating 2,000 requests of up to 2,000 x 20,000 cells costs
    no per-request alignment simulation; the likelihood arithmetic does not depend on the codes'
    correlation across taxa."""
    rng = np.random.default_rng(seed)
    out = {}
    for m in (4, 61):
        t = rng.integers(0, m, size=(max_taxa, max_patterns), dtype=np.uint8)
        t[rng.random((max_taxa, max_patterns)) < ambiguous] = m
        out[m] = t
    return out


def serving_problem(desc, masters):
    """Problem of one serving request: a Yule tree of desc["n_tips"] taxa, branch lengths
    Exp(mean 0.01), a general 4-state Q or a codon Q, desc["n_cat"] discrete-gamma categories
    (shape 0.5) and a view of desc["n_patterns"] patterns of the master tip matrix."""
    rng = np.random.default_rng(desc["seed"])
    N, P, m, C = desc["n_tips"], desc["n_patterns"], desc["n_states"], desc["n_cat"]
    parent, _ = yule_tree(N, rng)
    b = branch_lengths(parent, 0.01, rng)
    if m == 61:
        Q, pi = codon_Q(rng)
    else:
        Q, pi = random_general_Q(4, rng), dirichlet_freqs(4, rng)
    rates, cw = discrete_gamma(0.5, C)
    master = masters[m]
    off = int(rng.integers(0, master.shape[1] - P + 1))
    pr = make_problem(parent, np.zeros((0, 0), dtype=np.uint8), np.ones(P), Q, pi, rates, cw, b)
    pr["tip_states"] = master[:N, off:off + P]   # row-strided view, not copied
    return pr


def materialise_request(desc):
    return random_problem(desc["n_tips"], desc["n_patterns"], n_states=desc["n_states"],
                          n_cat=desc["n_cat"], seed=desc["seed"], b_mean=0.01)
