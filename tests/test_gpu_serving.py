"""The continuous-batching server: every request's result is the same bits alone (pg_eval on its
own handle) and in the mix (admitted among others on several streams, under arena pressure), the
plain one-slot path gives the same results, and failing requests fail alone."""
import numpy as np
import pytest

from paper_1905_12146_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def mix():
    masters = wl.serving_masters(max_taxa=300, max_patterns=3000, seed=1)
    descs = wl.serving_requests(14, seed=3, taxa=(20, 300), patterns=(100, 3000), p_codon=0.3)
    assert any(d["n_states"] == 61 for d in descs) and any(d["n_states"] == 4 for d in descs)
    return [wl.serving_problem(d, masters) for d in descs]


@pytest.fixture(scope="module")
def alone(ctx, mix):
    out = []
    for p in mix:
        h = ctx.upload(p)
        try:
            out.append(h.eval(p["b"], grad=True))
        finally:
            h.close()
    return out


def _same(res, ref):
    assert res["status"] == 0
    assert res["logL"] == ref["logL"]
    np.testing.assert_array_equal(res["grad"], ref["grad"])


@pytest.mark.parametrize("slots,arena_gb", [(4, 8), (1, 8), (6, 1.5)])
def test_results_identical_alone_and_in_the_mix(ctx, mix, alone, slots, arena_gb):
    """All requests submitted at once: slots = 1 is the plain path; 1.5 GB holds only a few of
    the larger requests at a time, so admission waits for memory."""
    from paper_1905_12146_gb300 import _native
    srv = _native.Server(ctx, max_inflight=slots, arena_bytes=int(arena_gb * 2 ** 30))
    try:
        tickets = [srv.submit(p) for p in mix]
        res = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    for r, a in zip(res, alone):
        _same(r, a)
    for r in res:
        assert r["submit_s"] <= r["start_s"] <= r["done_s"]
    if slots > 1:   # some request was admitted while another was still running
        spans = sorted((r["start_s"], r["done_s"]) for r in res)
        assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_served_results_match_the_oracle(ctx, mix, oracle_mod):
    from paper_1905_12146_gb300 import _native
    small = [p for p in mix if p["n_tips"] <= 120][:3]
    assert small
    srv = _native.Server(ctx, max_inflight=3, arena_bytes=2 ** 30)
    try:
        res = [srv.wait(t) for t in [srv.submit(p) for p in small]]
    finally:
        srv.close()
    for p, r in zip(small, res):
        dense = dict(p, tip_states=np.ascontiguousarray(p["tip_states"]))
        ref = oracle_mod.evaluate(dense, p["b"])
        assert abs(r["logL"] - ref.logL) <= 1e-6 * abs(ref.logL)
        assert np.abs(r["grad"] - ref.grad).max() <= 2e-4 * np.abs(ref.grad).max()


def test_oversize_and_invalid_requests_fail_alone(ctx, mix, alone):
    from paper_1905_12146_gb300 import _native
    big = wl.serving_problem({"n_tips": 300, "n_patterns": 3000, "n_states": 61, "n_cat": 4, "seed": 9},
                             wl.serving_masters(max_taxa=300, max_patterns=3000, seed=1))
    nt = sorted((i for i, p in enumerate(mix) if p["n_states"] == 4), key=lambda i: mix[i]["n_tips"])
    i_bad, i_ok = nt[0], nt[1]
    bad_b = mix[i_bad]["b"].copy()
    bad_b[0] = -1.0
    srv = _native.Server(ctx, max_inflight=2, arena_bytes=256 * 2 ** 20)
    try:
        t_big = srv.submit(big)
        t_bad = srv.submit(mix[i_bad], b=bad_b)
        t_ok = srv.submit(mix[i_ok])
        with pytest.raises(_native.PhyloGradError) as e:
            srv.wait(t_big)
        assert e.value.status == _native.PG_ERR_OOM
        with pytest.raises(_native.PhyloGradError) as e:
            srv.wait(t_bad)
        assert e.value.status == _native.PG_ERR_INVALID
        _same(srv.wait(t_ok), alone[i_ok])
    finally:
        srv.close()
