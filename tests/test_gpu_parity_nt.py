"""GPU parity of the 4-state path against the FP64 oracle, through the C ABI.

Tolerances (written here, derived in the design notes):
* logL: relative 1e-9, the stated target.  FP64 partials meet it everywhere.  FP32 partials meet
  it on the full-size nucleotide configuration (asserted there); on small problems one FP32
  rounding per internal node per site is by itself a noise of about
  2^-24 sqrt(n_internal * sum_p w_p^2), comparable to 1e-9 |logL|, so there the bound is
  max(1e-9 |logL|, 6 * 2^-24 * sqrt(n_internal * sum_p w_p^2));
* gradient: max-norm relative 1e-5, ||g - g*||_inf / ||g*||_inf;
* Hessian diagonal: max-norm relative 1e-4 (a difference of two FP32 site terms);
* per-site logL: absolute 6 * n_internal * 2^-24 (every internal node rounds each FP32 partial at
  most a handful of times; relative rounding adds linearly in log space in the worst case).
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

LOGL_RTOL = 1e-9
GRAD_RTOL = 1e-5
HESS_RTOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_12146_gb300 import _native, build
    build.build()
    c = _native.Context(0)
    yield c
    c.close()


def _site_atol(pr, precision):
    if precision == "fp64":
        return 1e-10
    return 6.0 * (pr["n_tips"] - 1) * 2.0 ** -24 + 1e-12


def _logl_tol(pr, ref_logL, precision):
    tol = LOGL_RTOL * abs(ref_logL) + 1e-12
    if precision == "fp32":
        noise = 2.0 ** -24 * np.sqrt((pr["n_tips"] - 1) * np.sum(pr["weights"] ** 2))
        tol = max(tol, 6.0 * noise)
    return tol


def _compare(ctx, oracle_mod, pr, hess=True, b=None, tile=None, precision="fp32"):
    from paper_1905_12146_gb300 import _native
    c = ctx if tile is None else _native.Context(0, patterns_per_tile=tile)
    h = c.upload(pr, precision)
    try:
        b = pr["b"] if b is None else b
        got = h.eval(b, grad=True, hess=hess, site=True)
        ref = oracle_mod.evaluate(pr, b)
    finally:
        h.close()
        if tile is not None:
            c.close()
    assert got["status"] == 0
    assert abs(got["logL"] - ref.logL) <= _logl_tol(pr, ref.logL, precision), (got["logL"], ref.logL)
    gscale = max(np.abs(ref.grad).max(), 1e-300)
    assert np.abs(got["grad"] - ref.grad).max() <= GRAD_RTOL * gscale
    root = wl.root_of(pr["parent"])
    assert got["grad"][root] == 0.0
    if pr["weights"].shape[0]:
        np.testing.assert_allclose(got["site_logL"], ref.site_logL, rtol=0, atol=_site_atol(pr, precision))
    if hess:
        hscale = max(np.abs(ref.hess).max(), 1e-300)
        assert np.abs(got["hess"] - ref.hess).max() <= HESS_RTOL * hscale
    return got, ref


def test_small_configuration_fp64(ctx, oracle_mod):
    """16 taxa, 500 patterns with integer weights, one category, general Q, FP64 partials:
    the plain FP64 method, so logL within 1e-9 relative (observed ~1e-15)."""
    pr = wl.config_small(seed=0)
    got, ref = _compare(ctx, oracle_mod, pr, precision="fp64")
    assert abs(got["logL"] - ref.logL) <= 1e-12 * abs(ref.logL)
    assert np.abs(got["grad"] - ref.grad).max() <= 1e-11 * np.abs(ref.grad).max()


@pytest.mark.parametrize("case", ["small", "cat4", "caterpillar", "two_taxa", "models", "zero_and_long", "wide"])
def test_fp64_latency_kernel_and_device_partials_kernel(ctx, oracle_mod, case):
    """FP64 problems evaluated alone run in the shared-memory latency kernel when a block's vectors
    fit; PG_FLAG_FP64_DEVICE_PARTIALS selects the kernel with the partials in device memory.  Both
    against the oracle at the FP64 bounds, and against each other (the same products, summed in
    another order)."""
    from paper_1905_12146_gb300 import _native
    pr = {"small": lambda: wl.config_small(seed=3),
          "cat4": lambda: wl.random_problem(60, 333, n_states=4, n_cat=4, seed=31, b_mean=0.05, ambiguous=0.03,
                                            weights="int"),
          "caterpillar": lambda: wl.random_problem(120, 200, n_states=4, n_cat=2, seed=32, tree="caterpillar",
                                                   b_mean=0.02, ambiguous=0.02),
          "two_taxa": lambda: wl.random_problem(2, 70, n_states=4, n_cat=3, seed=33, b_mean=0.3, ambiguous=0.2),
          "models": lambda: wl.random_problem(40, 257, n_states=4, n_cat=2, seed=34, n_models=3, relabel=True,
                                              ambiguous=0.05, weights="int"),
          "zero_and_long": lambda: wl.random_problem(30, 150, n_states=4, n_cat=2, seed=35, b_mean=0.05),
          "wide": lambda: wl.random_problem(24, 2400, n_states=4, n_cat=1, seed=36, b_mean=0.1, weights="int"),
          }[case]()
    b = pr["b"].copy()
    if case == "zero_and_long":
        b[::5] = 0.0
        b[2::9] = 20.0
        b[wl.root_of(pr["parent"])] = 0.0
    ref = oracle_mod.evaluate(pr, b)
    out = []
    for flags in (0, _native.PG_FLAG_FP64_DEVICE_PARTIALS):
        c = _native.Context(0, flags=flags)
        h = c.upload(pr, "fp64")
        try:
            got = h.eval(b, grad=True, hess=True, site=True)
        finally:
            h.close()
            c.close()
        assert got["status"] == 0
        assert abs(got["logL"] - ref.logL) <= 1e-12 * abs(ref.logL)
        assert np.abs(got["grad"] - ref.grad).max() <= 1e-11 * np.abs(ref.grad).max()
        assert np.abs(got["hess"] - ref.hess).max() <= 1e-10 * np.abs(ref.hess).max()
        np.testing.assert_allclose(got["site_logL"], ref.site_logL, rtol=0, atol=1e-10)
        assert got["grad"][wl.root_of(pr["parent"])] == 0.0
        out.append(got)
    a, d = out
    assert abs(a["logL"] - d["logL"]) <= 1e-13 * abs(d["logL"])
    assert np.abs(a["grad"] - d["grad"]).max() <= 1e-12 * np.abs(d["grad"]).max()
    np.testing.assert_allclose(a["site_logL"], d["site_logL"], rtol=0, atol=1e-12)


def test_small_configuration_fp32(ctx, oracle_mod):
    _compare(ctx, oracle_mod, wl.config_small(seed=0), precision="fp32")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("n_cat", [1, 2, 3, 4])
def test_rate_categories(ctx, oracle_mod, n_cat, precision):
    pr = wl.random_problem(60, 333, n_states=4, n_cat=n_cat, seed=100 + n_cat, b_mean=0.05,
                           ambiguous=0.03, weights="int")
    _compare(ctx, oracle_mod, pr, precision=precision)


@pytest.mark.parametrize("tile", [2, 7, 32, 100, 1024])
def test_tile_sizes_and_ragged_tail(ctx, oracle_mod, tile):
    pr = wl.random_problem(40, 1000 + 17, n_states=4, n_cat=4, seed=7, b_mean=0.02,
                           ambiguous=0.02)
    _compare(ctx, oracle_mod, pr, tile=tile)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_non_homogeneous_models_and_relabelled_nodes(ctx, oracle_mod, precision):
    pr = wl.random_problem(80, 257, n_states=4, n_cat=2, seed=8, n_models=3, relabel=True,
                           ambiguous=0.05, weights="int")
    _compare(ctx, oracle_mod, pr, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_caterpillar_tree(ctx, oracle_mod, precision):
    """Height N-1: one level per internal node."""
    pr = wl.random_problem(300, 200, n_states=4, n_cat=2, seed=9, tree="caterpillar",
                           b_mean=0.02, ambiguous=0.02)
    _compare(ctx, oracle_mod, pr, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_two_taxa(ctx, oracle_mod, precision):
    pr = wl.random_problem(2, 70, n_states=4, n_cat=3, seed=10, b_mean=0.3, ambiguous=0.2)
    _compare(ctx, oracle_mod, pr, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_long_branches_and_zero_lengths(ctx, oracle_mod, precision):
    pr = wl.random_problem(50, 120, n_states=4, n_cat=2, seed=11, b_mean=0.05)
    b = pr["b"].copy()
    b[::7] = 0.0
    b[3::11] = 25.0
    b[wl.root_of(pr["parent"])] = 0.0
    _compare(ctx, oracle_mod, pr, b=b, precision=precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_reversible_model(ctx, oracle_mod, precision):
    pr = wl.random_problem(100, 500, n_states=4, n_cat=4, seed=12, reversible=True,
                           b_mean=0.03, ambiguous=0.02)
    _compare(ctx, oracle_mod, pr, precision=precision)


def test_deep_underflow_fp32(ctx, oracle_mod):
    """Saturated JC69 tip branches on 700 taxa: L_p = 4^-N ~ 2^-1400, far below FP32 and FP64
    range; the per-node power-of-two rescaling must carry it."""
    rng = np.random.default_rng(13)
    parent, _ = wl.yule_tree(700, rng)
    b = rng.exponential(0.1, size=parent.shape[0])
    b[:700] = 60.0
    b[parent < 0] = 0.0
    tips = rng.integers(0, 5, size=(700, 64)).astype(np.uint8)
    pr = wl.make_problem(parent, tips, np.ones(64), wl.jc69_Q(), np.full(4, 0.25), np.ones(1),
                         np.ones(1), b)
    for precision in ("fp32", "fp64"):
        h = ctx.upload(pr, precision)
        got = h.eval(b, site=True)
        h.close()
        n_obs = (tips < 4).sum(axis=0)
        np.testing.assert_allclose(got["site_logL"], -n_obs * np.log(4.0), rtol=1e-6)


def test_empty_alignment(ctx):
    pr = wl.random_problem(10, 5, n_states=4, n_cat=2, seed=13)
    pr = dict(pr, tip_states=pr["tip_states"][:, :0], weights=pr["weights"][:0])
    h = ctx.upload(pr)
    got = h.eval(pr["b"], hess=True)
    h.close()
    assert got["logL"] == 0.0
    assert np.all(got["grad"] == 0.0) and np.all(got["hess"] == 0.0)


@pytest.mark.slow
def test_nucleotide_configuration_full_size(ctx, oracle_mod):
    """1,000 taxa, 10,000 patterns, 4 gamma categories, 2% ambiguous cells: every output, FP32
    partials, and logL within the stated 1e-9 relative."""
    pr = wl.config_nucleotide()
    got, ref = _compare(ctx, oracle_mod, pr, hess=False)
    rel = abs(got["logL"] - ref.logL) / abs(ref.logL)
    assert rel <= LOGL_RTOL
    gerr = np.abs(got["grad"] - ref.grad).max() / np.abs(ref.grad).max()
    print(f"\nconfig nucleotide: logL rel err {rel:.3e}, grad max-norm rel err {gerr:.3e}")


def test_batch_equals_single(ctx, oracle_mod):
    """A batched launch runs every level below the root in level kernels shared by the batch
    (a problem alone runs its narrow levels in the top kernel), so batch and single results differ
    by FP32 rounding order only: both meet the parity bounds against the oracle, and they agree
    with each other within the same bounds."""
    torch = pytest.importorskip("torch")
    probs = [wl.random_problem(20 + 7 * i, 100 + 31 * i, n_states=4, n_cat=1 + i % 4, seed=200 + i,
                               ambiguous=0.02) for i in range(6)]
    hs = [ctx.upload(p) for p in probs]
    dev = torch.device("cuda")
    bs = [torch.tensor(p["b"], device=dev) for p in probs]
    single = []
    for h, b in zip(hs, bs):
        lg = torch.zeros(1, dtype=torch.float64, device=dev)
        g = torch.zeros_like(b)
        hh = torch.zeros_like(b)
        h.eval_async(b, lg, g, hh)
        torch.cuda.synchronize()
        single.append((lg.clone(), g.clone(), hh.clone()))
    from paper_1905_12146_gb300 import _native
    lgs = torch.zeros(len(hs), dtype=torch.float64, device=dev)
    gs = [torch.zeros_like(b) for b in bs]
    hhs = [torch.zeros_like(b) for b in bs]
    _native.eval_batch_async(hs, bs, lgs, gs, hhs)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        ref = oracle_mod.evaluate(p, p["b"])
        tol = _logl_tol(p, ref.logL, "fp32")
        for lg, g, hh in ((lgs[i].item(), gs[i], hhs[i]), (single[i][0].item(), single[i][1], single[i][2])):
            assert abs(lg - ref.logL) <= tol
            assert np.abs(g.cpu().numpy() - ref.grad).max() <= GRAD_RTOL * np.abs(ref.grad).max()
            assert np.abs(hh.cpu().numpy() - ref.hess).max() <= HESS_RTOL * np.abs(ref.hess).max()
        assert abs(lgs[i].item() - single[i][0].item()) <= 2 * tol
        assert (gs[i] - single[i][1]).abs().max().item() <= 2 * GRAD_RTOL * np.abs(ref.grad).max()
    for h in hs:
        h.close()


def test_stream_and_device_pointers(ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    pr = wl.random_problem(64, 640, n_states=4, n_cat=4, seed=14, ambiguous=0.02)
    h = ctx.upload(pr)
    dev = torch.device("cuda")
    s = torch.cuda.Stream()
    b = torch.tensor(pr["b"], device=dev)
    lg = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros_like(b)
    site = torch.zeros(640, dtype=torch.float64, device=dev)
    s.wait_stream(torch.cuda.current_stream())
    h.eval_async(b, lg, g, None, site, stream=s)
    assert h.status() == 0
    ref = oracle_mod.evaluate(pr)
    assert abs(lg.item() - ref.logL) <= LOGL_RTOL * abs(ref.logL)
    assert np.abs(g.cpu().numpy() - ref.grad).max() <= GRAD_RTOL * np.abs(ref.grad).max()
    h.close()


def test_bad_branch_length_reported(ctx):
    from paper_1905_12146_gb300 import _native
    pr = wl.random_problem(10, 40, n_states=4, seed=15)
    h = ctx.upload(pr)
    b = pr["b"].copy()
    b[2] = -1.0
    with pytest.raises(_native.PhyloGradError) as e:
        h.eval(b)
    assert e.value.status == _native.PG_ERR_INVALID
    b[2] = np.nan
    with pytest.raises(_native.PhyloGradError):
        h.eval(b)
    assert h.eval(pr["b"])["status"] == 0   # status cleared, handle still usable
    h.close()


def test_impossible_site_reported(ctx):
    """A generator with a zero column makes a state unreachable: L_p = 0 -> PG_ERR_NUMERIC."""
    rng = np.random.default_rng(3)
    Q = wl.random_general_Q(4, rng, normalise=False)
    Q[:, 3] = 0.0
    np.fill_diagonal(Q, 0.0)
    np.fill_diagonal(Q, -Q.sum(axis=1))
    parent, _ = wl.yule_tree(6, rng)
    tips = np.zeros((6, 4), dtype=np.uint8)
    tips[0, 1] = 3
    pr = wl.make_problem(parent, tips, np.ones(4), Q, np.array([0.3, 0.3, 0.4, 0.0]), np.ones(1),
                         np.ones(1), wl.branch_lengths(parent, 0.1, rng))
    h = ctx.upload(pr)
    assert h.eval(pr["b"])["status"] == 5
    h.close()


def test_host_validation(ctx):
    from paper_1905_12146_gb300 import _native
    pr = wl.random_problem(8, 20, n_states=4, seed=16)
    bad = pr["parent"].copy()
    bad[0] = bad[1] = bad[2] = bad[3]
    for broken in (dict(pr, parent=bad),
                   dict(pr, root_freqs=pr["root_freqs"] * 2),
                   dict(pr, Q=pr["Q"] + 0.1),
                   dict(pr, weights=-pr["weights"]),
                   dict(pr, cat_weights=np.array([0.7]))):
        with pytest.raises(_native.PhyloGradError) as e:
            ctx.upload(broken)
        assert e.value.status == _native.PG_ERR_INVALID
    for unsupported, precision in ((wl.random_problem(5, 4, n_states=65, seed=1), "fp32"),   # > 64 states
                                   (wl.random_problem(5, 4, n_states=20, seed=1), "fp64")):  # FP64: 4 states
        with pytest.raises(_native.PhyloGradError) as e:
            ctx.upload(unsupported, precision)
        assert e.value.status == _native.PG_ERR_UNSUPPORTED


def test_budget_admission():
    from paper_1905_12146_gb300 import _native
    c = _native.Context(0, hbm_budget_bytes=1 << 20)
    with pytest.raises(_native.PhyloGradError) as e:
        c.upload(wl.random_problem(200, 2000, n_states=4, n_cat=4, seed=17))
    assert e.value.status == _native.PG_ERR_OOM
    c.close()


def test_branch_lengths_written_by_the_previous_launch(ctx):
    """Two evaluations back to back on one stream, the second taking as its branch lengths the
    gradient buffer the first one's reduction writes.  The second one's transition-matrix launch
    may start while that reduction runs (it stores its tables only after waiting for it, and reads
    b again then), so its results and status are those of the same evaluation from a copy of the
    buffer made after a synchronisation, bit for bit.  Four taxa whose four tips differ at every
    site, on branches of 1e-3: every branch carries a change in some most parsimonious history, so
    every gradient entry but the root's (0) is positive and the gradient is a valid set of branch
    lengths, while the zeros the buffer held before give P = I and a likelihood of 0."""
    torch = pytest.importorskip("torch")
    pr = wl.random_problem(4, 3000, n_states=4, n_cat=4, seed=23)
    rng = np.random.default_rng(5)
    pr["tip_states"] = np.ascontiguousarray(np.stack([rng.permutation(4) for _ in range(3000)], axis=1),
                                            dtype=np.uint8)
    pr["b"] = np.full_like(pr["b"], 1e-3)
    h = ctx.upload(pr)
    dev = torch.device("cuda")
    b0 = torch.tensor(pr["b"], device=dev)
    z = lambda n: torch.zeros(n, dtype=torch.float64, device=dev)   # noqa: E731
    bits = lambda x: x.view(torch.int64)                              # noqa: E731
    n = b0.numel()
    l1, g1 = z(1), z(n)
    h.eval_async(b0, l1, g1)
    torch.cuda.synchronize()
    assert h.status() == 0
    assert (g1[:-1] > 0).all().item() and g1[-1].item() == 0.0
    for _ in range(3):
        la, ga, lb, gb = z(1), z(n), z(1), z(n)
        h.eval_async(b0, la, ga)
        h.eval_async(ga, lb, gb)   # ga is written by the launch just before
        torch.cuda.synchronize()
        assert h.status() == 0 and np.isfinite(lb.item())
        assert torch.equal(bits(la), bits(l1)) and torch.equal(bits(ga), bits(g1))
        lc, gc = z(1), z(n)
        h.eval_async(ga.clone(), lc, gc)
        torch.cuda.synchronize()
        assert h.status() == 0
        assert torch.equal(bits(lb), bits(lc)) and torch.equal(bits(gb), bits(gc))
    h.close()


def test_phase_timing_modes(ctx):
    """Phase timing: mode 1 times every phase, mode 2 only the pre-order levels (the other fields
    stay 0), mode 3 those of every 8th evaluation; each counts the evaluations it timed; another
    mode is an invalid argument.  Timing changes no
    result bit."""
    torch = pytest.importorskip("torch")
    from paper_1905_12146_gb300 import _native
    pr = wl.random_problem(400, 2000, n_states=4, n_cat=4, seed=31)
    h = ctx.upload(pr)
    dev = torch.device("cuda")
    b = torch.tensor(pr["b"], device=dev)
    outs = []
    for mode in (1, 2, 3, 0):
        h.set_phase_timing(mode)
        lg, g = torch.zeros(1, dtype=torch.float64, device=dev), torch.zeros_like(b)
        for _ in range(9):
            h.eval_async(b, lg, g)
        torch.cuda.synchronize()
        pt = h.phase_times()
        outs.append((lg.clone(), g.clone()))
        if mode == 1:
            assert pt.evals == 9 and pt.pre_levels_ms > 0 and pt.post_levels_ms > 0 and pt.total_ms > 0
        elif mode in (2, 3):
            assert pt.evals == (9 if mode == 2 else 2) and pt.pre_levels_ms > 0   # mode 3: the 1st and 9th
            assert pt.post_levels_ms == 0 and pt.pmatrix_ms == 0 and pt.total_ms == 0
        else:
            assert pt.evals == 0
    for lg, g in outs[1:]:
        assert torch.equal(lg, outs[0][0]) and torch.equal(g, outs[0][1])
    with pytest.raises(_native.PhyloGradError) as e:
        h.set_phase_timing(4)
    assert e.value.status == _native.PG_ERR_INVALID
    assert h.status() == 0
    h.close()


@pytest.mark.parametrize("n_cat", [1, 2])
def test_single_problem_level_kernels_with_few_categories(ctx, oracle_mod, n_cat):
    """A single problem with one or two rate categories that runs its wide levels in the level
    kernels (cut 4-5 here): the cherry level's items cover four ranges of 256 patterns, and the
    pattern count leaves the last item with ranges past the last pattern.  Parity with the oracle,
    Hessian diagonal and per-site values included."""
    pr = wl.random_problem(500, 2500 + 37 * n_cat, n_states=4, n_cat=n_cat, seed=40 + n_cat, b_mean=0.05,
                           ambiguous=0.02)
    _compare(ctx, oracle_mod, pr)
