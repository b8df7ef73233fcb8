"""The forward/backward split, the torch.autograd.Functions and the random-effects clock chain rule,
against pg_eval, the FP64 oracle and central finite differences.

Tolerances as in the nucleotide parity tests: logL within 1e-9 relative (with the FP32 noise bound
on small problems), gradients within 1e-5 max-norm relative.  Finite differences are central with
h = 1e-6 on FP64 log-likelihoods (the oracle's, or the library's FP64-partial mode); their
truncation error is O(h^2) and their rounding error about c 2^-53 |logL| / h.  On the 12-taxon,
300-pattern clock problem that is far below 1e-6 relative, the bound used there; on the
5,000-pattern trees the bound is derived in the test.
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5
FD_RTOL = 1e-6
H = 1e-6


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.fixture(scope="module")
def ctx(torch):
    from paper_1905_12146_gb300 import _native, build
    build.build()
    c = _native.Context(0)
    yield c
    c.close()


def _logl_tol(pr, ref_logL, precision="fp32"):
    tol = 1e-9 * abs(ref_logL) + 1e-12
    if precision == "fp32":
        tol = max(tol, 6.0 * 2.0 ** -24 * np.sqrt((pr["n_tips"] - 1) * np.sum(pr["weights"] ** 2)))
    return tol


def _maxrel(got, ref):
    return np.abs(np.asarray(got) - np.asarray(ref)).max() / max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("n_tips,n_patterns,n_cat,precision", [
    (200, 3000, 4, "fp32"),      # level kernels + top kernel
    (1000, 10000, 4, "fp32"),    # the full nucleotide shape
    (40, 700, 2, "fp32"),        # fused kernel only
    (40, 700, 3, "fp64"),        # FP64 partials (the backward recomputes the post-order)
])
def test_forward_backward_equals_eval(torch, ctx, n_tips, n_patterns, n_cat, precision):
    """Forward then backward give the bits of one pg_eval_async; the gradient scale is exact."""
    pr = wl.random_problem(n_tips, n_patterns, n_cat=n_cat, seed=11, b_mean=0.02, ambiguous=0.02)
    h = ctx.upload(pr, precision)
    try:
        dev = torch.device("cuda")
        b = torch.tensor(pr["b"], device=dev)
        n = b.shape[0]
        l0 = torch.zeros(1, dtype=torch.float64, device=dev)
        g0, h0 = torch.zeros(n, dtype=torch.float64, device=dev), torch.zeros(n, dtype=torch.float64, device=dev)
        h.eval_async(b, l0, g0, h0)
        l1 = torch.zeros(1, dtype=torch.float64, device=dev)
        g1, h1 = torch.zeros_like(g0), torch.zeros_like(h0)
        scale = torch.tensor([2.5], dtype=torch.float64, device=dev)
        h.forward_async(b, l1)
        h.backward_async(scale, g1, h1)
        g2 = torch.zeros_like(g0)
        h.backward_async(None, g2)   # a second backward on the same forward
        torch.cuda.synchronize()
        assert h.status() == 0
        assert l1.item() == l0.item()
        assert torch.equal(g1, 2.5 * g0)
        assert torch.equal(g2, g0)
        assert torch.equal(h1, h0)
    finally:
        h.close()


def test_backward_without_forward_is_rejected(torch, ctx):
    from paper_1905_12146_gb300 import _native
    pr = wl.random_problem(8, 50, seed=1)
    h = ctx.upload(pr)
    try:
        g = torch.zeros(pr["parent"].shape[0], dtype=torch.float64, device="cuda")
        with pytest.raises(_native.PhyloGradError) as e:
            h.backward_async(None, g)
        assert e.value.status == _native.PG_ERR_INVALID
    finally:
        h.close()


def test_batch_forward_backward_equals_batch_eval(torch, ctx):
    from paper_1905_12146_gb300 import _native
    probs = [wl.random_problem(30 + 7 * i, 400 + 90 * i, n_cat=1 + i % 4, seed=20 + i, b_mean=0.03)
             for i in range(6)]
    hs = [ctx.upload(p) for p in probs]
    try:
        dev = torch.device("cuda")
        bs = [torch.tensor(p["b"], device=dev) for p in probs]
        l0 = torch.zeros(len(hs), dtype=torch.float64, device=dev)
        g0 = [torch.zeros_like(b) for b in bs]
        _native.eval_batch_async(hs, bs, l0, g0)
        l1 = torch.zeros_like(l0)
        g1 = [torch.zeros_like(b) for b in bs]
        scale = torch.arange(1, len(hs) + 1, dtype=torch.float64, device=dev)
        _native.forward_batch_async(hs, bs, l1)
        _native.backward_batch_async(hs, scale, g1)
        torch.cuda.synchronize()
        assert torch.equal(l0, l1)
        for i in range(len(hs)):
            assert torch.equal(g1[i], (i + 1) * g0[i])
    finally:
        for h in hs:
            h.close()


def test_autograd_tree_loglik_against_oracle(torch, ctx, oracle_mod):
    from paper_1905_12146_gb300 import autograd as ag
    pr = wl.random_problem(120, 2000, n_cat=4, seed=5, b_mean=0.02, ambiguous=0.02)
    h = ctx.upload(pr)
    try:
        b = torch.tensor(pr["b"], device="cuda")[None].requires_grad_(True)
        logL = ag.tree_loglik(b, [h])
        (3.0 * logL.sum()).backward()
        ag.check_status([h])
        ref = oracle_mod.evaluate(pr, pr["b"])
        assert abs(logL.item() - ref.logL) <= _logl_tol(pr, ref.logL)
        assert _maxrel(b.grad[0].cpu().numpy(), 3.0 * ref.grad) <= GRAD_RTOL
    finally:
        h.close()


def test_autograd_recomputes_a_replaced_forward(torch, ctx, oracle_mod):
    """Two forwards on one handle, then the first one's backward: the partials of the first are
    recomputed before its pre-order pass."""
    from paper_1905_12146_gb300 import autograd as ag
    pr = wl.random_problem(60, 900, n_cat=2, seed=6, b_mean=0.03)
    h = ctx.upload(pr)
    try:
        b1 = torch.tensor(pr["b"], device="cuda")[None].requires_grad_(True)
        b2 = (1.7 * torch.tensor(pr["b"], device="cuda"))[None].requires_grad_(True)
        l1 = ag.tree_loglik(b1, [h])
        l2 = ag.tree_loglik(b2, [h])
        l1.sum().backward()
        l2.sum().backward()
        ref1 = oracle_mod.evaluate(pr, pr["b"])
        ref2 = oracle_mod.evaluate(pr, 1.7 * pr["b"])
        assert _maxrel(b1.grad[0].cpu().numpy(), ref1.grad) <= GRAD_RTOL
        assert _maxrel(b2.grad[0].cpu().numpy(), ref2.grad) <= GRAD_RTOL
    finally:
        h.close()


def _oracle_clock_logl(oracle_mod, pr, eps, mu, t):
    par = pr["parent"]
    b = np.zeros(par.shape[0])
    nz = par >= 0
    b[nz] = mu * eps[nz] * (t[nz] - t[par[nz]])
    return oracle_mod.evaluate(pr, b).logL


def test_clock_chain_rule_against_oracle_finite_differences(torch, ctx, oracle_mod):
    """d logL / d(eps, mu, t) through the clock kernels and the FP64 backward, against central
    differences of the oracle's FP64 logL in every parameter (sign and index of each term)."""
    from paper_1905_12146_gb300 import autograd as ag
    rng = np.random.default_rng(9)
    parent, node_time = wl.yule_tree(12, rng)
    eps = rng.lognormal(0.0, 0.5, size=parent.shape[0])
    nz = parent >= 0
    mu = 0.05 / float(np.mean(eps[nz] * (node_time[nz] - node_time[parent[nz]])))
    b = np.zeros(parent.shape[0])
    b[nz] = mu * eps[nz] * (node_time[nz] - node_time[parent[nz]])
    Q = wl.random_general_Q(4, rng)
    pi = wl.dirichlet_freqs(4, rng)
    tips = wl.simulate_alignment(parent, b, Q, pi, np.ones(1), np.ones(1), 300, rng)
    pr = wl.make_problem(parent, tips, np.ones(300), Q, pi, np.ones(1), np.ones(1), b, node_time=node_time)
    h = ctx.upload(pr, "fp64")
    try:
        dev = torch.device("cuda")
        te = torch.tensor(eps, device=dev)[None].requires_grad_(True)
        tm = torch.tensor([mu], dtype=torch.float64, device=dev).requires_grad_(True)
        tt = torch.tensor(node_time, device=dev)[None].requires_grad_(True)
        logL = ag.tree_loglik(ag.clock_branch_lengths(te, tm, tt, [h]), [h])
        logL.sum().backward()
        ag.check_status([h])
        root = wl.root_of(parent)
        fd_eps, fd_t = np.zeros_like(eps), np.zeros_like(node_time)
        for i in range(parent.shape[0]):
            if i != root:
                e1, e2 = eps.copy(), eps.copy()
                e1[i] += H
                e2[i] -= H
                fd_eps[i] = (_oracle_clock_logl(oracle_mod, pr, e1, mu, node_time) -
                             _oracle_clock_logl(oracle_mod, pr, e2, mu, node_time)) / (2 * H)
            t1, t2 = node_time.copy(), node_time.copy()
            t1[i] += H
            t2[i] -= H
            fd_t[i] = (_oracle_clock_logl(oracle_mod, pr, eps, mu, t1) -
                       _oracle_clock_logl(oracle_mod, pr, eps, mu, t2)) / (2 * H)
        fd_mu = (_oracle_clock_logl(oracle_mod, pr, eps, mu * (1 + H), node_time) -
                 _oracle_clock_logl(oracle_mod, pr, eps, mu * (1 - H), node_time)) / (2 * H * mu)
        assert _maxrel(te.grad[0].cpu().numpy(), fd_eps) <= FD_RTOL
        assert _maxrel(tt.grad[0].cpu().numpy(), fd_t) <= FD_RTOL
        assert abs(tm.grad.item() - fd_mu) <= FD_RTOL * abs(fd_mu)
        assert te.grad[0, root].item() == 0.0
    finally:
        h.close()


@pytest.fixture(scope="module")
def clock_batch():
    return wl.config_clock_batch()


def test_differentiation_batch_against_oracle(torch, ctx, oracle_mod, clock_batch):
    """64 trees x 300 taxa x 5,000 patterns, one category: the batched clock -> logL -> backward
    through autograd; every tree's logL, d/d eps, d/d mu and d/d t against the oracle's FP64
    logL and branch gradient carried through the clock."""
    from paper_1905_12146_gb300 import autograd as ag
    probs = clock_batch
    hs = [ctx.upload(p) for p in probs]
    try:
        dev = torch.device("cuda")
        eps = torch.tensor(np.stack([p["eps"] for p in probs]), device=dev).requires_grad_(True)
        mu = torch.tensor([p["mu"] for p in probs], dtype=torch.float64, device=dev).requires_grad_(True)
        t = torch.tensor(np.stack([p["node_time"] for p in probs]), device=dev).requires_grad_(True)
        logL = ag.tree_loglik(ag.clock_branch_lengths(eps, mu, t, hs), hs)
        logL.sum().backward()
        ag.check_status(hs)
        got_l = logL.detach().cpu().numpy()
        for i, p in enumerate(probs):
            par = p["parent"]
            nz = par >= 0
            b = np.zeros(par.shape[0])
            b[nz] = p["mu"] * p["eps"][nz] * (p["node_time"][nz] - p["node_time"][par[nz]])
            np.testing.assert_allclose(b, p["b"], rtol=1e-13, atol=0)
            ref = oracle_mod.evaluate(p, b)
            assert abs(got_l[i] - ref.logL) <= _logl_tol(p, ref.logL), i
            dt = np.where(nz, p["node_time"] - p["node_time"][np.maximum(par, 0)], 0.0)
            g = np.where(nz, ref.grad, 0.0)
            r = p["mu"] * p["eps"]
            ref_eps = p["mu"] * dt * g
            ref_mu = float(np.sum(p["eps"] * dt * g))
            ref_t = r * g
            np.subtract.at(ref_t, par[nz], (r * g)[nz])
            assert _maxrel(eps.grad[i].cpu().numpy(), ref_eps) <= GRAD_RTOL, i
            assert _maxrel(t.grad[i].cpu().numpy(), ref_t) <= GRAD_RTOL, i
            assert abs(mu.grad[i].item() - ref_mu) <= GRAD_RTOL * np.abs(p["eps"] * dt * g).sum(), i
    finally:
        for h in hs:
            h.close()


def test_differentiation_batch_finite_differences_all_branches(torch, ctx, clock_batch):
    """Central differences (h = 1e-6) on every branch of one of the 64 trees against the FP32
    batched backward's gradient.  The step is taken in log b (positive parameters are
    log-transformed, Section 3), so the difference approximates b_i dlogL/db_i: an absolute step
    of 1e-6 on a branch of length 4e-5 would carry a truncation error (h^2 / 6) f3 of several
    units, f3 the third derivative (sites whose likelihood is proportional to b give f3 = 2 / b^3).
    What remains is rounding: the two FP64 logL values (|logL| ~ 1.5e5) differ by about
    c 2^-53 |logL| (c ~ 100 for 5,000 patterns x 300 taxa), divided by 2h."""
    from paper_1905_12146_gb300 import autograd as ag
    p = clock_batch[0]
    hs = [ctx.upload(q) for q in clock_batch[:8]]
    h64 = ctx.upload(p, "fp64")
    try:
        dev = torch.device("cuda")
        b = torch.tensor(np.stack([q["b"] for q in clock_batch[:8]]), device=dev).requires_grad_(True)
        ag.tree_loglik(b, hs).sum().backward()
        ag.check_status(hs)
        got = p["b"] * b.grad[0].cpu().numpy()
        root = wl.root_of(p["parent"])
        logL = h64.eval(p["b"], grad=False)["logL"]
        fd = np.zeros_like(p["b"])
        for i in range(p["b"].shape[0]):
            if i == root:
                continue
            bp, bm = p["b"].copy(), p["b"].copy()
            bp[i] *= np.exp(H)
            bm[i] *= np.exp(-H)
            fd[i] = (h64.eval(bp, grad=False)["logL"] - h64.eval(bm, grad=False)["logL"]) / (2 * H)
        tol = GRAD_RTOL * np.abs(fd).max() + 100 * 2.0 ** -53 * abs(logL) / (2 * H)
        assert np.abs(got - fd).max() <= tol, (np.abs(got - fd).max(), tol)
    finally:
        h64.close()
        for h in hs:
            h.close()
