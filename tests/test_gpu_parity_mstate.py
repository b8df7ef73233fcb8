"""GPU parity of the general-state path (61 sense codons, 20 amino acids) against the FP64 oracle.

Stated error.  The transition tables D = P - I are formed by uniformisation (FP64 powers of the
uniformised chain and FP64 Poisson weights summed in FP32), the partials are FP32 and the tensor-core
products three-pass TF32 with the identity part of P x kept out of the (truncating) tensor-core
accumulation.  Every internal node then perturbs a site's likelihood by independent FP32 roundings:
sums of m products (random-walk growth, sqrt(m)) plus a few roundings of the product and scale
(a constant), so over n_int internal nodes the site logL error is bounded by
16 sqrt(n_int) (sqrt(m) + 1) 2^-24.  Measured on the problems below (both kernel families), the
largest site error is 5.4 sqrt(n_int) (sqrt(m) + 1) 2^-24: the bound holds with a margin of 3.
logL is bounded by the weighted sum of the site bounds.  The gradient bound is the benchmark spec's
1e-5 of the max-norm (largest measured error 1.9e-6, a margin of 5); the Hessian diagonal's is 2e-5
(largest measured 2.4e-6, a margin of 8).
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

M_GRAD_RTOL = 1e-5
M_HESS_RTOL = 2e-5


@pytest.fixture(scope="module", params=["tensor", "simt"])
def ctx(request):
    """Both kernel families of the general-state path: tcgen05 (default) and CUDA-core FP32."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_12146_gb300 import _native, build
    build.build()
    c = _native.Context(0, flags=0 if request.param == "tensor" else _native.PG_FLAG_SIMT_MSTATE)
    c.kind = request.param
    yield c
    c.close()


def _maxrel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def _site_atol(pr):
    m = pr["Q"].shape[-1]
    n_int = pr["parent"].shape[0] - pr["n_tips"]
    return 16.0 * np.sqrt(n_int) * (np.sqrt(m) + 1.0) * 2.0 ** -24


def _logl_atol(pr, weights=None):
    w = pr["weights"] if weights is None else weights
    return _site_atol(pr) * float(np.sum(np.abs(w))) + 1e-12


def _check(ctx, oracle_mod, pr, hess=True, label=""):
    h = ctx.upload(pr)
    try:
        got = h.eval(pr["b"], grad=True, hess=hess, site=True)
        plain = h.eval(pr["b"], grad=True, hess=False, site=True) if hess else got
    finally:
        h.close()
    ref = oracle_mod.evaluate(pr, pr["b"])
    # the evaluation without the Hessian runs its own pre-order kernel: same bounds
    assert plain["status"] == 0
    assert abs(plain["logL"] - ref.logL) <= _logl_atol(pr)
    assert _maxrel(plain["grad"], ref.grad) <= M_GRAD_RTOL
    print(f"{ctx.kind} {label} (no Hessian): grad {_maxrel(plain['grad'], ref.grad):.2e}")
    el = abs(got["logL"] - ref.logL) / abs(ref.logL)
    eg = _maxrel(got["grad"], ref.grad)
    es = np.abs(got["site_logL"] - ref.site_logL).max() if pr["weights"].shape[0] else 0.0
    eh = _maxrel(got["hess"], ref.hess) if hess else 0.0
    print(f"{ctx.kind} {label}: logL rel {el:.2e}  grad {eg:.2e}  site abs {es:.2e}  hess {eh:.2e}  "
          f"site / bound {es / _site_atol(pr):.2f}  logL abs / bound {abs(got['logL'] - ref.logL) / _logl_atol(pr):.3f}")
    assert got["status"] == 0
    assert abs(got["logL"] - ref.logL) <= _logl_atol(pr)
    assert eg <= M_GRAD_RTOL
    assert es <= _site_atol(pr)
    if hess:
        assert eh <= M_HESS_RTOL
    assert got["grad"][wl.root_of(pr["parent"])] == 0.0
    return got, ref


@pytest.mark.parametrize("n_tips,n_patterns,n_cat,seed", [
    (3, 40, 1, 1), (12, 130, 4, 2), (40, 300, 2, 3), (25, 64, 3, 4), (17, 1, 1, 5),
])
def test_codon_against_oracle(ctx, oracle_mod, n_tips, n_patterns, n_cat, seed):
    """61-state reversible codon model: several pattern tiles with a ragged tail, one pattern,
    a three-taxon tree."""
    pr = wl.random_problem(n_tips, n_patterns, n_states=61, n_cat=n_cat, seed=seed, b_mean=0.05,
                           ambiguous=0.03)
    _check(ctx, oracle_mod, pr, label=f"codon N={n_tips} P={n_patterns} C={n_cat}")


def test_codon_caterpillar_and_models(ctx, oracle_mod):
    """Deep (caterpillar) tree, two codon models on different branches, relabelled nodes."""
    pr = wl.random_problem(30, 200, n_states=61, n_cat=2, seed=7, tree="caterpillar", n_models=2, b_mean=0.1)
    _check(ctx, oracle_mod, pr, label="codon caterpillar 2 models")
    pr = wl.random_problem(30, 150, n_states=61, n_cat=1, seed=8, relabel=True, b_mean=0.1)
    _check(ctx, oracle_mod, pr, hess=False, label="codon relabelled")


@pytest.mark.parametrize("m", [2, 3, 5, 20, 33, 64])
def test_other_state_counts(ctx, oracle_mod, m):
    pr = wl.random_problem(20, 257, n_states=m, n_cat=2, seed=30 + m, reversible=True, b_mean=0.1,
                           ambiguous=0.05)
    _check(ctx, oracle_mod, pr, label=f"m={m}")


@pytest.mark.parametrize("m", [20, 61])
def test_non_reversible_general_state_space(ctx, oracle_mod, m):
    """A general (non-reversible) generator with a root distribution that is not stationary."""
    rng = np.random.default_rng(40 + m)
    pr = wl.random_problem(15, 180, n_states=m, n_cat=2, seed=40 + m, b_mean=0.1, ambiguous=0.03)
    pr["Q"] = wl.random_general_Q(m, rng)[None]
    pr["root_freqs"] = wl.dirichlet_freqs(m, rng)
    _check(ctx, oracle_mod, pr, label=f"non-reversible m={m}")


def test_short_branches_and_unlikely_sites(ctx, oracle_mod):
    """Codon tips drawn independently of the tree on very short branches: the site likelihoods
    rest on multi-step transition probabilities of order t^3, which must stay positive and
    relatively accurate."""
    rng = np.random.default_rng(77)
    pr = wl.random_problem(40, 300, n_states=61, n_cat=4, seed=77, b_mean=0.002)
    pr["tip_states"] = rng.integers(0, 61, size=pr["tip_states"].shape).astype(np.uint8)
    _check(ctx, oracle_mod, pr, label="codon random tips, short branches")


def test_codon_forward_backward_equals_eval(ctx):
    import torch
    pr = wl.random_problem(40, 333, n_states=61, n_cat=4, seed=9, b_mean=0.05)
    h = ctx.upload(pr)
    try:
        dev = torch.device("cuda")
        b = torch.tensor(pr["b"], device=dev)
        l0 = torch.zeros(1, dtype=torch.float64, device=dev)
        g0 = torch.zeros_like(b)
        h.eval_async(b, l0, g0)
        l1, g1 = torch.zeros_like(l0), torch.zeros_like(b)
        scale = torch.tensor([-0.5], dtype=torch.float64, device=dev)
        h.forward_async(b, l1)
        h.backward_async(scale, g1)
        torch.cuda.synchronize()
        assert h.status() == 0
        assert l1.item() == l0.item()
        assert torch.equal(g1, -0.5 * g0)
    finally:
        h.close()


@pytest.fixture(scope="module")
def codon_full():
    return wl.config_codon()


def test_codon_full_size_sampled_sites(ctx, oracle_mod, codon_full):
    """500 taxa x 3,000 codon patterns x 4 categories, as timed: the per-site logL of 60 sampled
    patterns against the oracle run on those patterns alone, and the gradient of an evaluation
    whose weights are zero except on the sampled patterns against the oracle's gradient of that
    sub-alignment (same shapes and launches as the full evaluation)."""
    pr = dict(codon_full)
    P = pr["weights"].shape[0]
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(P, 60, replace=False))
    h = ctx.upload(pr)
    try:
        full = h.eval(pr["b"], grad=True, site=True)
        w = np.zeros(P)
        w[idx] = pr["weights"][idx]
        masked = dict(pr, weights=w)
    finally:
        h.close()
    hm = ctx.upload(masked)
    try:
        part = hm.eval(pr["b"], grad=True, site=True)
    finally:
        hm.close()
    sub = dict(pr, tip_states=pr["tip_states"][:, idx], weights=pr["weights"][idx])
    ref = oracle_mod.evaluate(sub, pr["b"])
    es = np.abs(full["site_logL"][idx] - ref.site_logL).max()
    eg = _maxrel(part["grad"], ref.grad)
    el = abs(part["logL"] - ref.logL) / abs(ref.logL)
    print(f"codon full size: site abs {es:.2e}  masked logL rel {el:.2e}  masked grad {eg:.2e}")
    assert full["status"] == 0 and part["status"] == 0
    assert es <= _site_atol(pr)
    assert abs(part["logL"] - ref.logL) <= _logl_atol(pr, sub["weights"])
    assert eg <= M_GRAD_RTOL
    np.testing.assert_array_equal(part["site_logL"], full["site_logL"])


def _with_partial_tips(pr, m, rng, frac=0.15):
    """Partially observed tips (Section 2.1): the IUPAC ambiguity sets and base-call likelihoods
    for nucleotides, random subsets with graded entries for larger state spaces."""
    if m == 4:
        table = wl.iupac_nucleotide_partials(error=0.03)
    else:
        table = np.where(rng.random((12, m)) < 0.3, rng.uniform(0.2, 1.0, (12, m)), 0.0)
        table[np.arange(12), rng.integers(0, m, 12)] = 1.0
    pr = dict(pr, tip_partials=table)
    pr["tip_states"] = wl.make_partially_observed(pr["tip_states"], frac, table, rng)
    return pr


@pytest.mark.parametrize("m", [4, 20, 61])
def test_partially_observed_tips(ctx, oracle_mod, m):
    """Tip partial vectors, indicator codes and missing data mixed in every tile (a 4-state
    problem with tip vectors runs on this path); 300 patterns = two full tiles and a ragged one."""
    rng = np.random.default_rng(60 + m)
    pr = wl.random_problem(24, 300, n_states=m, n_cat=2, seed=60 + m, b_mean=0.1, ambiguous=0.05)
    pr = _with_partial_tips(pr, m, rng)
    codes = pr["tip_states"]
    assert ((codes >= m) & (codes < m + len(pr["tip_partials"]))).any() and (codes == wl.MISSING).any()
    _check(ctx, oracle_mod, pr, label=f"partial tips m={m}")


def test_partially_observed_tips_host_validation(ctx):
    from paper_1905_12146_gb300 import _native
    rng = np.random.default_rng(70)
    pr = _with_partial_tips(wl.random_problem(8, 40, n_states=4, seed=70), 4, rng)
    for table in (-pr["tip_partials"], np.zeros_like(pr["tip_partials"]),
                  np.full_like(pr["tip_partials"], np.nan), np.full_like(pr["tip_partials"], np.inf)):
        with pytest.raises(_native.PhyloGradError) as e:
            ctx.upload(dict(pr, tip_partials=table))
        assert e.value.status == _native.PG_ERR_INVALID
    with pytest.raises(_native.PhyloGradError) as e:   # FP64 partials: the 4-state path only
        ctx.upload(pr, "fp64")
    assert e.value.status == _native.PG_ERR_UNSUPPORTED


@pytest.mark.parametrize("m", [4, 61])
def test_partially_observed_tips_beyond_fp32_range(ctx, oracle_mod, m):
    """Tip partial vectors are only required to be finite: rows with entries beyond the FP32 range,
    rows whose sum exceeds it and rows below its normal range are held scaled by exact powers of
    two, whose exponents are added back to the site log-likelihoods (the gradient and Hessian
    diagonal are ratios in which they cancel)."""
    rng = np.random.default_rng(72 + m)
    pr = _with_partial_tips(wl.random_problem(12, 160, n_states=m, n_cat=2, seed=72 + m, b_mean=0.1), m, rng,
                            frac=0.3)
    table = pr["tip_partials"].copy()
    scale = np.ones(table.shape[0])
    scale[0::4] = 1e39                       # entries beyond FLT_MAX
    scale[1::4] = 3.0e38 / table.max(1)[1::4]   # largest entry near FLT_MAX, row sum beyond it
    scale[2::4] = 1e-41                      # every entry below the FP32 normal range
    pr["tip_partials"] = table * scale[:, None]
    _check(ctx, oracle_mod, pr, label=f"scaled tip rows m={m}")
    # the same problem with the unscaled rows differs in logL by the scales' logs alone
    plain = oracle_mod.evaluate(dict(pr, tip_partials=table), pr["b"])
    scaled = oracle_mod.evaluate(pr, pr["b"])
    codes = pr["tip_states"].astype(np.int64)
    sel = (codes >= m) & (codes < m + table.shape[0])
    shift = np.where(sel, np.log(scale[np.clip(codes - m, 0, table.shape[0] - 1)]), 0.0).sum(0)
    np.testing.assert_allclose(scaled.site_logL - plain.site_logL, shift, rtol=1e-12, atol=1e-9)


def test_codon_transition_tables_against_expm(ctx):
    """The device's transition matrices (uniformisation: FP64 powers and Poisson weights, FP32 sums)
    entry by entry against scipy's expm, for the codon generator over b r from 1e-4 to 5.  A 2-taxon
    tree whose second branch has length 0 (P = I) has site likelihood pi_y2 P(b)[y2, y1], so the 61^2
    patterns (y2, y1) expose every entry of P(b) through the site log-likelihoods.  Off the diagonal
    P = D, small probabilities stay relatively accurate (bound 1e-5; measured 2.5e-6 at b r = 5).  The
    diagonal is 1 + D in FP32, whose rounding is absolute: about 2^-24 of 1, however small P_ii is at
    long branches (bound 16 2^-24; measured 1.5e-7 at b r = 5, where the smallest P_ii is 4e-3)."""
    import scipy.linalg as sla
    rng = np.random.default_rng(91)
    m = 61
    Q, _ = wl.codon_Q(rng)
    pi = wl.dirichlet_freqs(m, rng)
    y2, y1 = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
    tips = np.stack([y1.ravel(), y2.ravel()]).astype(np.uint8)
    pr = wl.make_problem(np.array([2, 2, -1], dtype=np.int32), tips, np.ones(m * m), Q, pi,
                         np.array([1.0]), np.array([1.0]), np.array([0.1, 0.0, 0.0]))
    h = ctx.upload(pr)
    try:
        for t in (1e-4, 1e-3, 1e-2, 0.1, 0.5, 1.0, 2.0, 5.0):
            got = h.eval(np.array([t, 0.0, 0.0]), grad=False, site=True)
            assert got["status"] == 0
            Pd = (np.exp(got["site_logL"]) / pi[y2.ravel()]).reshape(m, m)   # Pd[y2, y1] = P[y2, y1]
            Pe = sla.expm(Q * t)
            off = ~np.eye(m, dtype=bool)
            rel_off = np.abs(Pd[off] - Pe[off]) / Pe[off]
            abs_diag = np.abs(np.diag(Pd) - np.diag(Pe))
            print(f"{ctx.kind} t={t:g}: max rel error off-diagonal {rel_off.max():.2e}, abs diagonal {abs_diag.max():.2e}, "
                  f"smallest entry {Pe[off].min():.1e}")
            assert (Pd > 0).all()
            assert rel_off.max() <= 1e-5 and abs_diag.max() <= 16 * 2.0 ** -24
    finally:
        h.close()
