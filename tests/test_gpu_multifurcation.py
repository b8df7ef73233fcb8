"""Trees with multifurcations through the library against the FP64 oracle.

The library evaluates a node of degree d > 2 as a chain of d - 2 added nodes joined by branches of
length 0; callers pass and receive arrays of their own n nodes.  The oracle takes the product over
the wider sibling set directly (Sections 2.3-2.4).  Parity bounds are those of the binary paths:
4 states FP32 max(1e-9 |logL|, 6 2^-24 sqrt(n_int sum w^2)) for logL, 1e-5 of the max-norm for the
gradient, 1e-4 for the Hessian diagonal; FP64 1e-12; general state spaces the stated bounds of the
general path (site logL 16 sqrt(n_int) (sqrt(m) + 1) 2^-24, gradient 1e-5, Hessian 2e-5).
"""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_12146_gb300 import _native, build
    build.build()
    return _native


def _maxrel(got, ref):
    return np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-300)


def _bounds(pr, precision, logL):
    """(absolute logL bound, gradient and Hessian max-norm relative bounds)."""
    m = pr["Q"].shape[-1]
    n_int = pr["parent"].shape[0] - pr["n_tips"]
    w = pr["weights"]
    if precision == "fp64":
        return 1e-12 * abs(logL), 1e-11, 1e-10
    if m == 4:
        return max(1e-9 * abs(logL), 6 * 2.0 ** -24 * np.sqrt(n_int * np.sum(w ** 2))), 1e-5, 1e-4
    site = 16.0 * np.sqrt(n_int) * (np.sqrt(m) + 1.0) * 2.0 ** -24
    return site * np.sum(np.abs(w)), 1e-5, 2e-5


def _check(got, ref, pr, precision, label):
    lb, gb, hb = _bounds(pr, precision, ref.logL)
    el = abs(got["logL"] - ref.logL)
    eg = _maxrel(got["grad"], ref.grad)
    eh = _maxrel(got["hess"], ref.hess) if got.get("hess") is not None else 0.0
    print(f"{label}: logL abs {el:.2e} (bound {lb:.1e})  grad {eg:.2e}  hess {eh:.2e}")
    assert got["status"] == 0
    assert el <= lb
    assert eg <= gb
    assert eh <= hb
    assert got["grad"][wl.root_of(pr["parent"])] == 0.0


@pytest.mark.parametrize("m,precision,flags,n_tips,n_collapse,n_pat,seed", [
    (4, "fp32", 0, 60, 15, 700, 1),     # level kernels, top kernel, a few degree >= 4 nodes
    (4, "fp64", 0, 40, 10, 300, 2),     # fused FP64 kernel
    (61, "fp32", 0, 25, 6, 260, 3),     # tensor-core kernels
    (61, "fp32", 1, 25, 6, 260, 3),     # CUDA-core kernels
    (20, "fp32", 0, 30, 8, 150, 4),
])
def test_multifurcating_tree_against_oracle(native, oracle_mod, m, precision, flags, n_tips, n_collapse, n_pat, seed):
    pr = wl.multifurcating_problem(n_tips, n_pat, n_collapse, n_states=m, n_cat=4 if m == 4 else 2, seed=seed,
                                   b_mean=0.05 if m == 4 else 0.1, ambiguous=0.03)
    n = pr["parent"].shape[0]
    assert n == 2 * n_tips - 1 - n_collapse and np.bincount(pr["parent"][pr["parent"] >= 0]).max() >= 3
    ctx = native.Context(0, flags=flags)
    h = ctx.upload(pr, precision)
    try:
        assert h.info().n_nodes == n
        got = h.eval(pr["b"], grad=True, hess=True, site=True)
    finally:
        h.close()
        ctx.close()
    ref = oracle_mod.evaluate(pr)
    assert got["grad"].shape == (n,)
    _check(got, ref, pr, precision, f"m={m} {precision} flags={flags} N={n_tips} n={n}")


def test_star_tree(native, oracle_mod):
    """One internal node holding every tip: N - 2 added nodes in a chain."""
    base = wl.random_problem(12, 300, n_states=4, n_cat=2, seed=5, b_mean=0.2, ambiguous=0.05)
    parent = np.full(13, 12, dtype=np.int32)
    parent[12] = -1
    b = np.random.default_rng(5).exponential(0.2, 13)
    b[12] = 0.0
    pr = dict(base, parent=parent, b=b, n_tips=12, node_time=None)
    ctx = native.Context(0)
    h = ctx.upload(pr, "fp32")
    try:
        got = h.eval(pr["b"], grad=True, hess=True)
    finally:
        h.close()
        ctx.close()
    _check(got, oracle_mod.evaluate(pr), pr, "fp32", "star tree")


def test_multifurcating_async_batch_forward_backward(native, oracle_mod):
    """Device entry points with arrays of the caller's n nodes: nothing is written past them, the
    batch mixes binary and multifurcating problems, and forward + backward equal one evaluation."""
    import torch
    dev = torch.device("cuda")
    probs = [wl.multifurcating_problem(50, 500, 12, n_states=4, n_cat=2, seed=11, b_mean=0.05),
             wl.random_problem(30, 400, n_states=4, n_cat=2, seed=12, b_mean=0.05),
             wl.multifurcating_problem(20, 200, 5, n_states=61, n_cat=2, seed=13, b_mean=0.1)]
    ctx = native.Context(0)
    hs = [ctx.upload(p, "fp32") for p in probs]
    try:
        guard = 7.25
        bs = [torch.tensor(p["b"], device=dev) for p in probs]
        gs = [torch.full((p["parent"].shape[0] + 8,), guard, dtype=torch.float64, device=dev) for p in probs]
        logL = torch.zeros(len(probs), dtype=torch.float64, device=dev)
        native.eval_batch_async(hs, bs, logL, d_grad=gs)
        torch.cuda.synchronize()
        for i, (p, h) in enumerate(zip(probs, hs)):
            n = p["parent"].shape[0]
            assert h.status() == 0
            assert torch.all(gs[i][n:] == guard)        # nothing written past the caller's nodes
            ref = oracle_mod.evaluate(p)
            got = {"logL": logL[i].item(), "grad": gs[i][:n].cpu().numpy(), "hess": None, "status": 0}
            _check(got, ref, p, "fp32", f"batch entry {i} (n={n})")
        # single-problem device calls on the first (multifurcating) problem
        p, h = probs[0], hs[0]
        n = p["parent"].shape[0]
        l0 = torch.zeros(1, dtype=torch.float64, device=dev)
        g0 = torch.full((n + 8,), guard, dtype=torch.float64, device=dev)
        hh = torch.full((n + 8,), guard, dtype=torch.float64, device=dev)
        h.eval_async(bs[0], l0, g0, hh)
        l1 = torch.zeros(1, dtype=torch.float64, device=dev)
        g1 = torch.full((n + 8,), guard, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        h.forward_async(bs[0], l1)
        h.backward_async(None, g1)
        torch.cuda.synchronize()
        assert h.status() == 0
        assert torch.all(g0[n:] == guard) and torch.all(hh[n:] == guard) and torch.all(g1[n:] == guard)
        assert l1.item() == l0.item()
        assert torch.equal(g1[:n], g0[:n])
        ref = oracle_mod.evaluate(p)
        _check({"logL": l0.item(), "grad": g0[:n].cpu().numpy(), "hess": hh[:n].cpu().numpy(), "status": 0},
               ref, p, "fp32", "eval_async")
    finally:
        for h in hs:
            h.close()
        ctx.close()


def test_multifurcating_request_through_the_server(native, oracle_mod):
    pr = wl.multifurcating_problem(40, 600, 10, n_states=4, n_cat=3, seed=21, b_mean=0.05)
    ctx = native.Context(0)
    srv = native.Server(ctx, max_inflight=2)
    try:
        t = srv.submit(pr, grad=True, hess=True)
        t2 = srv.submit(wl.random_problem(30, 300, n_states=4, n_cat=1, seed=22))
        got = srv.wait(t)
        assert srv.wait(t2)["status"] == 0
    finally:
        srv.close()
        ctx.close()
    _check(got, oracle_mod.evaluate(pr), pr, "fp32", "served")


def test_multifurcation_host_validation(native):
    pr = wl.multifurcating_problem(10, 20, 3, n_states=4, seed=31)
    ctx = native.Context(0)
    try:
        bad = pr["parent"].copy()
        root = wl.root_of(bad)
        kids = np.bincount(bad[bad >= 0], minlength=bad.shape[0])
        k = int([x for x in np.flatnonzero(kids == 2) if x != root][0])   # leave it one child
        c = int(np.flatnonzero(bad == k)[0])
        bad[c] = root
        with pytest.raises(native.PhyloGradError) as e:
            ctx.upload(dict(pr, parent=bad))
        assert e.value.status == native.PG_ERR_INVALID
        bad = pr["parent"].copy()
        bad[0] = 1                                # a tip as a parent
        with pytest.raises(native.PhyloGradError) as e:
            ctx.upload(dict(pr, parent=bad))
        assert e.value.status == native.PG_ERR_INVALID
        with pytest.raises(native.PhyloGradError) as e:   # the allocation-free entry point: binary only
            native.eval_noalloc(pr, pr["b"], "fp32")
        assert e.value.status == native.PG_ERR_UNSUPPORTED
        h = ctx.upload(pr)
        try:
            import torch
            dev = torch.device("cuda")
            n = pr["parent"].shape[0]
            z = torch.zeros(n, dtype=torch.float64, device=dev)
            mu = torch.ones(1, dtype=torch.float64, device=dev)
            with pytest.raises(native.PhyloGradError) as e:   # the clock takes binary trees
                native.clock_lengths_async([h], [z], mu, [z], [z])
            assert e.value.status == native.PG_ERR_UNSUPPORTED
        finally:
            h.close()
    finally:
        ctx.close()
