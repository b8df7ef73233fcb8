#!/usr/bin/env python3
"""Throughput of logL + branch-gradient evaluations on one GB300 (or N, as independent replicas).

Workload (default): the nucleotide configuration -- a 1,000-taxon Yule tree with b ~ Exp(0.01), a
general non-reversible 4x4 generator, 4 discrete-gamma rate categories (shape 0.5) and 10,000
site patterns simulated down the tree with 2% all-ones ambiguous tip cells; one evaluation is
logL plus the 1,998 branch gradients (FP32 partials, FP64 transition matrices and sums).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One JSON line is printed by rank 0.  ``value`` is evaluations/s with every input resident in HBM
(device branch lengths, device outputs), timed with CUDA events; ``e2e`` is the same metric through
the blocking host-pointer call (branch lengths copied from pinned host memory, logL and gradient
copied back each step).  ``roofline`` is for the dominant kernel (the pre-order level kernels,
timed by the library's events around them on every 8th evaluation of the timed region);
``phases`` splits an evaluation by phase in a separate pass with an event at every phase boundary;
``cpu_baseline`` is the FP64 CPU oracle on a bounded sample of the same workload.
``--impl reference`` times that oracle alone (there is no reference GPU implementation).

Rank 0 then adds measured objects (skipped with ``--no-extras``): ``small`` (per-call latency of
the 16-taxon, 500-pattern FP64 configuration, p50 / p99), ``codon`` (500 taxa x 3,000 codon
patterns x 4 categories on the tensor-core kernels, with its error against the FP64 oracle), ``differentiation`` (the 64-tree clock
batch through the torch.autograd.Functions), ``inference`` (L-BFGS branch rates, analytic gradient
against finite differences), ``hmc`` (HMC over the branch rates, identity mass against the
Hessian-adapted diagonal mass, effective samples per second) and ``serving``
(``--serving-requests`` Poisson requests through the continuous-batching server against the
one-request-at-a-time plain path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "logL+branch-gradient evals/s"
UNIT = "evals/s"
WORKLOAD = ("nucleotide: 1,000-taxon Yule tree, b~Exp(0.01), non-reversible 4x4 Q, 4 gamma "
            "categories (shape 0.5), 10,000 simulated patterns, 2% ambiguous tips")


def _rank_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _max_over_ranks(seconds: float, dist, device):
    """Slowest rank's time (the job takes as long as its slowest replica); identity alone."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_throughput(units_per_rank: int, seconds: float, world: int, dist, device):
    """Whole-job throughput of replicas: every rank processed units_per_rank units of its own
    (weak scaling, no data-path collective); value = all ranks' units / the slowest rank's time."""
    slowest = _max_over_ranks(seconds, dist, device)
    return world * units_per_rank / slowest, slowest


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def _kernel_hash(read=None):
    """Hash of what the pre-order level kernel is built from: the whole of pg_levels.cu and the
    headers it includes, and the nvcc architecture and code-generation flags.  ``read(name) ->
    bytes`` reads a source file (default: the tree)."""
    from paper_1905_12146_gb300 import build as _build
    if read is None:
        def read(name):
            with open(os.path.join(ROOT, "paper_1905_12146_gb300", "csrc", name), "rb") as f:
                return f.read()
    h = hashlib.sha256()
    for name in ("pg_levels.cu", "pg_device.cuh", "pg_internal.cuh"):
        h.update(read(name))
    h.update(" ".join(_build.ARCH + _build.FLAGS).encode())
    return h.hexdigest()[:16]


def _traffic_from_profile():
    """DRAM bytes per evaluation of the pre-order level kernels from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pre_level_kernel_nucleotide.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    kv = {}
    for ln in lines:
        if ln.startswith("- ") and ":" in ln:
            k, v = ln[2:].split(":", 1)
            kv[k.strip()] = v.strip().strip("`")
    if kv.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    try:
        return float(kv["dram_bytes_per_eval"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.2)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        # under load: samples in the upper half of the observed range
        hi = sorted(sm)[len(sm) // 2:]
        return {"sm_mhz": statistics.median(hi), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _cpu_baseline(problem, seconds: float = 12.0):
    """The FP64 oracle on the host cores on a bounded sample of the workload (the first patterns
    of the alignment), scaled to evaluations/s of the full workload; the single-thread figure
    beside it."""
    from oracle import oracle
    oracle.build()
    P = problem["weights"].shape[0]
    sample = min(P, 1000)
    t0 = time.perf_counter()
    oracle.evaluate(problem, patterns=slice(0, sample))
    t1 = time.perf_counter()
    per = t1 - t0
    reps = max(1, min(20, int(seconds / 2 / max(per, 1e-3))))
    t0 = time.perf_counter()
    for _ in range(reps):
        ref = oracle.evaluate(problem, patterns=slice(0, sample))
    per = (time.perf_counter() - t0) / reps
    single = per * P / sample
    from oracle.parallel import OraclePool
    pool = OraclePool(problem)
    try:
        big = min(P, sample * pool.cores)
        pool.evaluate(0, big)   # workers started and warm
        t0 = time.perf_counter()
        preps = max(1, min(20, int(seconds / 2 / max(per * big / sample / pool.cores, 1e-3))))
        for _ in range(preps):
            pool.evaluate(0, big)
        pper = (time.perf_counter() - t0) / preps
    finally:
        pool.close()
    full = pper * P / big
    return {"value": 1.0 / full, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
            "sample": f"{big} of {P} patterns split over {pool.cores} processes, {preps} evaluations "
                      f"(FP64), time scaled by {P / big:g} to the full alignment",
            "seconds_per_full_eval": full,
            "single_thread": {"value": 1.0 / single, "cores": 1, "seconds_per_full_eval": single,
                              "sample": f"{sample} of {P} patterns, {reps} evaluations"}}, ref, sample


def _stated_error(ctx, problem, ref, sample, device, steps: int = 10):
    """Error against the FP64 oracle of the same call on the sampled patterns (weights of the
    others set to zero), for the FP32 path that ``value`` times and for the library's FP64 path,
    and the FP64 path's evaluations/s on the full workload (a floor: FP64 partials, every level in
    the fused kernel)."""
    import numpy as np
    import torch

    masked = dict(problem, weights=np.where(np.arange(problem["weights"].shape[0]) < sample, problem["weights"], 0.0))
    gmax = float(np.abs(ref.grad).max())
    out = {"reference": "FP64 oracle on the first %d patterns" % sample}
    for prec in ("fp32", "fp64"):
        h = ctx.upload(masked, prec)
        try:
            r = h.eval(problem["b"], grad=True)
        finally:
            h.close()
        out[prec] = {"logL_rel": abs(r["logL"] - ref.logL) / abs(ref.logL),
                     "grad_maxnorm_rel": float(np.abs(r["grad"] - ref.grad).max()) / gmax}
    h = ctx.upload(problem, "fp64")
    dev = torch.device("cuda", device)
    n = problem["parent"].shape[0]
    b = torch.tensor(problem["b"], device=dev)
    lg = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros(n, dtype=torch.float64, device=dev)
    try:
        for _ in range(3):
            h.eval_async(b, lg, g)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            h.eval_async(b, lg, g)
        e1.record()
        torch.cuda.synchronize(dev)
        out["fp64_path"] = {"ms_per_eval": e0.elapsed_time(e1) / steps,
                            "evals_per_s": 1e3 * steps / e0.elapsed_time(e1), "status": h.status()}
    finally:
        h.close()
    return out


def run_reference(args):
    rank, world, _ = _rank_env()
    if world > 1 and rank != 0:
        return 0
    from oracle import oracle
    from paper_1905_12146_gb300 import workloads
    oracle.build()
    from oracle.parallel import OraclePool
    pr = workloads.config_nucleotide()
    P = pr["weights"].shape[0]
    pool = OraclePool(pr)   # the oracle on every host core, before any timing
    try:
        # size each step so that warm-up + timed steps take about two minutes in total
        t0 = time.perf_counter()
        oracle.evaluate(pr, patterns=slice(0, 100))
        per_pattern = (time.perf_counter() - t0) / 100 / pool.cores
        budget = 120.0 / max(1, args.steps + args.warmup)
        sample = int(max(16, min(P, budget / max(per_pattern, 1e-6))))
        for _ in range(args.warmup):
            pool.evaluate(0, sample)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.evaluate(0, sample)
        elapsed = time.perf_counter() - t0
    finally:
        pool.close()
    full = elapsed / args.steps * P / sample
    value = 1.0 / full
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * full,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_tips": 1000, "n_patterns": P, "n_categories": 4,
                   "n_states": 4},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                         "sample": f"{sample} of {P} patterns per step split over {pool.cores} processes, "
                                   "scaled to the full alignment (FP64)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


SERVING = ("serving: Poisson arrivals of logL+gradient requests, taxa U{50..2000}, patterns "
           "U{500..20000}, 4 states (80%) or 61 codon states (20%), 1-4 gamma categories, Yule trees, "
           "b~Exp(0.01), tip rows drawn from seeded master matrices; admitted by device-arena budget")


def _serving(n_requests: int, device: int):
    """The serving configuration: saturated throughput of the plain path (one request at a time)
    and of continuous batching, then Poisson arrivals at 0.5, 0.7 and 0.9 of the continuous path's
    saturated throughput (and the plain path at 0.7 of it) with p50 / p99 latency (completion minus
    submission)."""
    import numpy as np

    from paper_1905_12146_gb300 import _native, workloads

    t0 = time.perf_counter()
    masters = workloads.serving_masters()
    descs = workloads.serving_requests(n_requests, seed=5)
    probs = [workloads.serving_problem(d, masters) for d in descs]
    gen_s = time.perf_counter() - t0
    ctx = _native.Context(device)

    def run(slots, rate=None, seed=7):
        srv = _native.Server(ctx, max_inflight=slots)
        gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(probs)) if rate else np.zeros(len(probs))
        t_next = time.perf_counter()
        tickets = []
        for p, g in zip(probs, gaps):
            t_next += g
            while True:
                dt = t_next - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.0005))
            tickets.append(srv.submit(p))
        res = [srv.wait(t) for t in tickets]
        srv.close()
        lat = np.array([r["done_s"] - r["submit_s"] for r in res]) * 1e3
        span = max(r["done_s"] for r in res) - min(r["submit_s"] for r in res)
        bad = sum(1 for r in res if r["status"] != 0)
        return {"evals_per_s": len(res) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "failed": bad,
                "offered_per_s": rate}

    out = {"workload": SERVING, "requests": n_requests, "codon_requests": sum(d["n_states"] == 61 for d in descs),
           "generation_s": gen_s, "unit": "evals/s, ms"}
    out["saturated_plain"] = run(1)
    out["saturated_continuous"] = run(8)
    sat = out["saturated_continuous"]["evals_per_s"]
    out["poisson"] = [dict(load=f, continuous=run(8, f * sat, seed=11 + i)) for i, f in enumerate((0.5, 0.7, 0.9))]
    out["poisson"][1]["plain"] = run(1, 0.7 * sat, seed=12)
    ctx.close()
    return out


def _differentiation(device: int, steps: int = 30, warmup: int = 3):
    """The differentiation batch: 64 trees x 300 taxa x 5,000 patterns, one category; one step is
    the clock branch lengths, the batched forward (post-order) and the autograd backward (pre-order
    gradient kernels and the clock chain rule)."""
    import numpy as np
    import torch

    from paper_1905_12146_gb300 import _native, autograd, workloads

    probs = workloads.config_clock_batch()
    ctx = _native.Context(device)
    hs = [ctx.upload(p) for p in probs]
    dev = torch.device("cuda", device)
    eps = torch.tensor(np.stack([p["eps"] for p in probs]), device=dev).requires_grad_(True)
    mu = torch.tensor([p["mu"] for p in probs], dtype=torch.float64, device=dev).requires_grad_(True)
    t = torch.tensor(np.stack([p["node_time"] for p in probs]), device=dev).requires_grad_(True)

    def step():
        eps.grad = mu.grad = t.grad = None
        autograd.tree_loglik(autograd.clock_branch_lengths(eps, mu, t, hs), hs).sum().backward()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    autograd.check_status(hs)
    ms = e0.elapsed_time(e1) / steps
    nbytes = sum(h.info().stream_bytes for h in hs)
    for h in hs:
        h.close()
    ctx.close()
    return {"workload": "64 Yule trees x 300 taxa x 5,000 patterns, 1 category, clock b = mu eps dt",
            "ms_per_step": ms, "evals_per_s": len(probs) / (ms * 1e-3), "unit": "tree evals/s",
            "algorithmic_bytes_per_step": nbytes, "achieved_gbs": nbytes / (ms * 1e-3) / 1e9}


def _inference(device: int):
    """The shape of the paper's Table 1: maximum-likelihood branch rates by L-BFGS with the
    analytic gradient against central finite differences, on a 104-taxon Yule tree (206 rates, as
    the paper's smallest example) with 1,000 simulated patterns.  FP64 partials (as the paper's
    implementation): with FP32 partials a central difference at h = 1e-6 is dominated by rounding
    (~1e-7 |logL| / 2h)."""
    import numpy as np

    from paper_1905_12146_gb300 import _native, inference, workloads

    pr = workloads.config_clock_batch(seed=31, n_trees=1, n_tips=104, n_patterns=1000)[0]
    ctx = _native.Context(device)
    h = ctx.upload(pr, "fp64")
    par = pr["parent"]
    theta0 = np.zeros(par.shape[0])
    theta0[par >= 0] = np.log(pr["mu"])
    out = {"workload": "104-taxon Yule tree, 206 branch rates, 1,000 simulated patterns, 1 category, "
                       "FP64 partials; L-BFGS (history 10, strong Wolfe) until |change| < 1e-9",
           "rates": int((par >= 0).sum())}
    # one-time set-up (CUDA module loading of the optimiser's and the library's kernels) outside
    # the timings
    inference.rate_mle(h, pr["node_time"], theta0, "analytic", max_iter=500, tolerance_change=1e-9)
    inference.rate_mle(h, pr["node_time"], theta0, "numeric", max_iter=2)
    for method in ("analytic", "numeric"):
        r = inference.rate_mle(h, pr["node_time"], theta0, method, max_iter=500, tolerance_change=1e-9)
        out[method] = {"seconds": r["seconds"], "iterations": r["iterations"], "logL": r["logL"],
                       "objective_evaluations": r["objective_evaluations"], "forward_passes": r["forward_passes"]}
    a, n = out["analytic"], out["numeric"]
    out["speedup_per_iteration"] = (n["seconds"] / max(n["iterations"], 1)) / (a["seconds"] / max(a["iterations"], 1))
    out["speedup_total"] = n["seconds"] / a["seconds"]
    h.close()
    ctx.close()
    return out


def _hmc(device: int, n_warm: int = 150, n_keep: int = 300, n_leapfrog: int = 10):
    """HMC over the 206 branch rates of the 104-taxon clock problem (the inference object's
    workload, FP64 partials), random-effects prior with psi = 0.5, from the prior mean: identity
    mass against the diagonal mass adapted to the Hessian (Section 3.2.1).  Both chains adapt the
    step size during the first n_warm iterations (discarded).  Reported: effective samples per
    second (min and median over the rates) of the kept iterations, acceptance, gradient
    evaluations."""
    import numpy as np

    from paper_1905_12146_gb300 import _native, hmc, workloads

    pr = workloads.config_clock_batch(seed=31, n_trees=1, n_tips=104, n_patterns=1000)[0]
    ctx = _native.Context(device)
    h = ctx.upload(pr, "fp64")
    out = {"workload": "104-taxon Yule tree, 206 branch rates, 1,000 simulated patterns, FP64 partials; "
                       f"{n_warm} warm-up + {n_keep} kept iterations, {n_leapfrog} leapfrog steps"}
    try:
        for name, adapt in (("identity_mass", False), ("hessian_mass", True)):
            tg = hmc.ClockTarget(h, pr["parent"], pr["node_time"], pr["mu"], 0.5)
            theta0 = np.full(tg.dim, tg.m)
            tg.logp_grad(theta0)   # one-time set-up outside the timing
            r = hmc.hmc(tg, theta0, n_iter=n_warm + n_keep, eps=0.02, n_leapfrog=n_leapfrog, adapt_mass=adapt,
                        k=10, adapt_eps_until=n_warm, seed=7)
            x = r["samples"][n_warm:]
            neff = np.array([hmc.ess(x[:, i]) for i in range(tg.dim)])
            sec_keep = r["seconds"] * n_keep / (n_warm + n_keep)
            out[name] = {"seconds": r["seconds"], "acceptance": float(r["accepted"][n_warm:].mean()),
                         "eps": r["eps"], "gradient_evaluations": r["gradient_evaluations"],
                         "ess_min": float(neff.min()), "ess_median": float(np.median(neff)),
                         "ess_per_s_min": float(neff.min() / sec_keep),
                         "ess_per_s_median": float(np.median(neff) / sec_keep)}
    finally:
        h.close()
        ctx.close()
    out["speedup_min_ess_per_s"] = out["hessian_mass"]["ess_per_s_min"] / max(out["identity_mass"]["ess_per_s_min"], 1e-30)
    return out


SMALL = ("small FP64: 16-taxon Yule tree, b~Exp(0.05), non-reversible 4x4 Q, Dirichlet root "
         "frequencies, 500 patterns with integer weights 1-5, 1 category; logL + 30 branch gradients")


def _small(device: int, calls: int = 2000, warmup: int = 50):
    """The small configuration (the plain FP64 method): per-call latency over ``calls`` calls of
    pg_eval (host arrays, copies and synchronisation included), pg_eval_async (device arrays; the
    device time between CUDA events on the stream around each call, and the host time from the
    call to the stream's completion) and pg_eval_noalloc (host arrays, nothing allocated), with the
    FP64 oracle's single-thread time for the same problem beside them.  Host times include the
    Python/ctypes call overhead (about 1-3 us)."""
    import numpy as np
    import torch

    from oracle import oracle
    from paper_1905_12146_gb300 import _native, workloads

    pr = workloads.config_small(seed=0)
    n = pr["parent"].shape[0]
    lib = _native.load()
    ctx = _native.Context(device)
    h = ctx.upload(pr, "fp64")
    dev = torch.device("cuda", device)
    b_host = np.ascontiguousarray(pr["b"])
    out_l, out_g = np.zeros(1), np.zeros(n)

    def pct(us):
        us = np.asarray(us)
        return {"p50_us": float(np.percentile(us, 50)), "p99_us": float(np.percentile(us, 99)),
                "mean_us": float(us.mean()), "calls": int(us.size)}

    res = {"workload": SMALL, "unit": "us per call"}
    # pg_eval: host arrays
    bp, lp, gp = b_host.ctypes.data, out_l.ctypes.data, out_g.ctypes.data
    for _ in range(warmup):
        lib.pg_eval(h._ptr, bp, lp, gp, None, None)
    t = []
    for _ in range(calls):
        t0 = time.perf_counter_ns()
        st = lib.pg_eval(h._ptr, bp, lp, gp, None, None)
        t.append((time.perf_counter_ns() - t0) / 1e3)
        if st != 0:
            raise SystemExit(f"pg_eval failed with status {st}")
    res["pg_eval"] = pct(t)
    # pg_eval_async: device arrays, per-call events
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    b = torch.tensor(pr["b"], device=dev)
    lg = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros(n, dtype=torch.float64, device=dev)
    args = (h._ptr, b.data_ptr(), lg.data_ptr(), g.data_ptr(), None, None, sp)
    for _ in range(warmup):
        lib.pg_eval_async(*args)
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(calls)]
    t = []
    for e0, e1 in evs:
        t0 = time.perf_counter_ns()
        e0.record(stream)
        lib.pg_eval_async(*args)
        e1.record(stream)
        stream.synchronize()
        t.append((time.perf_counter_ns() - t0) / 1e3)
    res["pg_eval_async_device"] = pct([1e3 * e0.elapsed_time(e1) for e0, e1 in evs])
    res["pg_eval_async_host"] = pct(t)
    res["async_status"] = h.status()
    h.close()
    ctx.close()
    # pg_eval_noalloc: host arrays, fixed scratch (the problem's validation and level planning are
    # part of every call)
    import ctypes
    pst, _keep = _native.problem_struct(pr, "fp64")
    pref = ctypes.byref(pst)
    for _ in range(warmup):
        lib.pg_eval_noalloc(pref, bp, lp, gp, None, None, None)
    t = []
    for _ in range(calls):
        t0 = time.perf_counter_ns()
        st = lib.pg_eval_noalloc(pref, bp, lp, gp, None, None, None)
        t.append((time.perf_counter_ns() - t0) / 1e3)
        if st != 0:
            raise SystemExit(f"pg_eval_noalloc failed with status {st}")
    res["pg_eval_noalloc"] = pct(t)
    # the oracle, single thread, the same problem
    oracle.build()
    reps = 20
    oracle.evaluate(pr)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.evaluate(pr)
    res["oracle_single_thread_us"] = (time.perf_counter() - t0) / reps * 1e6
    return res


def _codon_error(ctx, pr, n_sample: int = 24, seed: int = 0):
    """Error of the codon evaluation against the FP64 oracle on sampled patterns: the per-site logL
    of a full evaluation at the sampled patterns, and logL and gradient of an evaluation whose
    weights are zero except at the sampled patterns, against the oracle on that sub-alignment."""
    import numpy as np

    from oracle import oracle
    oracle.build()
    P = pr["weights"].shape[0]
    idx = np.sort(np.random.default_rng(seed).choice(P, n_sample, replace=False))
    h = ctx.upload(pr)
    try:
        full = h.eval(pr["b"], grad=False, site=True)
    finally:
        h.close()
    w = np.zeros(P)
    w[idx] = pr["weights"][idx]
    hm = ctx.upload(dict(pr, weights=w))
    try:
        part = hm.eval(pr["b"], grad=True)
    finally:
        hm.close()
    t0 = time.perf_counter()
    ref = oracle.evaluate(dict(pr, tip_states=pr["tip_states"][:, idx], weights=pr["weights"][idx]), pr["b"])
    gmax = float(np.abs(ref.grad).max())
    return {"reference": f"FP64 oracle on {n_sample} sampled patterns ({time.perf_counter() - t0:.1f} s)",
            "site_logL_abs_max": float(np.abs(full["site_logL"][idx] - ref.site_logL).max()),
            "logL_rel": abs(part["logL"] - ref.logL) / abs(ref.logL),
            "grad_maxnorm_rel": float(np.abs(part["grad"] - ref.grad).max()) / gmax,
            "status": [full["status"], part["status"]]}


def _codon(device: int, steps: int = 20, warmup: int = 3, error: bool = True):
    """The codon configuration: 500 taxa x 3,000 patterns x 4 categories, 61 states, tensor-core
    kernels (three-pass TF32, FP32 accumulation)."""
    import torch

    from paper_1905_12146_gb300 import _native, workloads

    pr = workloads.config_codon()
    ctx = _native.Context(device)
    h = ctx.upload(pr)
    dev = torch.device("cuda", device)
    b = torch.tensor(pr["b"], device=dev)
    lg = torch.zeros(1, dtype=torch.float64, device=dev)
    g = torch.zeros_like(b)
    for _ in range(warmup):
        h.eval_async(b, lg, g)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        h.eval_async(b, lg, g)
    e1.record()
    torch.cuda.synchronize(dev)
    st = h.status()
    ms = e0.elapsed_time(e1) / steps
    info = h.info()
    h.close()
    out = {"workload": "codon: 500-taxon Yule tree, 61-state codon Q (omega 0.3), 4 categories, 3,000 patterns",
           "ms_per_eval": ms, "evals_per_s": 1e3 / ms, "status": st,
           "algorithmic_bytes": info.stream_bytes, "achieved_gbs": info.stream_bytes / (ms * 1e-3) / 1e9,
           "useful_tflops": info.flops / (ms * 1e-3) / 1e12,
           "precision": "FP32 partials; three-pass TF32 tensor-core products with FP32 accumulation; "
                        "transition tables by uniformisation: FP64 powers and Poisson weights, FP32 sums"}
    if error:
        out["error"] = _codon_error(ctx, pr)
    ctx.close()
    return out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_1905_12146_gb300 import _native, workloads

    rank, world, local = _rank_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the library has no CPU path)")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    pr = workloads.config_nucleotide()
    ctx = _native.Context(local)
    h = ctx.upload(pr, "fp32")
    info = h.info()
    dev = torch.device("cuda", local)
    n = pr["parent"].shape[0]
    b = torch.tensor(pr["b"], device=dev)
    logL = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        h.eval_async(b, logL, grad, stream=stream)
    torch.cuda.synchronize(dev)
    if h.status() != 0:
        raise SystemExit(f"evaluation failed with status {h.status()}")

    # timed region: device-resident inputs and outputs, CUDA events on the launching stream; the
    # library's events bracket the pre-order levels of every 8th evaluation (mode 3), since an event
    # at every phase boundary (mode 1) would end the programmatic launch overlap there, and each
    # timed event stalls the stream for a few microseconds
    h.set_phase_timing(3)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clocks:
        start.record(stream)
        for _ in range(args.steps):
            h.eval_async(b, logL, grad, stream=stream)
        stop.record(stream)
        torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    ms = start.elapsed_time(stop)
    pt = h.phase_times()
    h.set_phase_timing(False)
    status = h.status()
    value, seconds = _job_throughput(args.steps, ms / 1e3, world, dist, dev)
    ms_per_step = seconds * 1e3 / args.steps

    # the per-phase split, from a separate untimed pass with an event at every phase boundary
    h.set_phase_timing(1)
    for _ in range(max(20, args.steps // 8)):
        h.eval_async(b, logL, grad, stream=stream)
    torch.cuda.synchronize(dev)
    pt_all = h.phase_times()
    h.set_phase_timing(False)

    # end to end: the blocking host-pointer call, pinned host buffers, copies inside the region
    b_host = torch.tensor(pr["b"]).pin_memory()
    out_logL = torch.zeros(1, dtype=torch.float64).pin_memory()
    out_grad = torch.zeros(n, dtype=torch.float64).pin_memory()
    lib = _native.load()
    e2e_steps = max(1, args.steps // 2)
    for _ in range(2):
        lib.pg_eval(h._ptr, b_host.data_ptr(), out_logL.data_ptr(), out_grad.data_ptr(), None, None)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = lib.pg_eval(h._ptr, b_host.data_ptr(), out_logL.data_ptr(), out_grad.data_ptr(), None, None)
        if st != 0:
            raise SystemExit(f"pg_eval failed with status {st}")
    e2e_value, _ = _job_throughput(e2e_steps, time.perf_counter() - t0, world, dist, dev)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 + 8 * n}

    peak, peak_kind = _peaks()
    pre_ms = pt.pre_levels_ms / max(pt.evals, 1)
    pre_gbs = pt.pre_levels_bytes / (pre_ms * 1e-3) / 1e9 if pre_ms > 0 else None
    traffic = _traffic_from_profile()
    roofline = {"bound": "hbm", "kernel": "pre_level_kernel (pre-order levels, all launches of one "
                                           "evaluation)",
                "achieved": pre_gbs, "peak": peak, "unit": "GB/s",
                "frac": (pre_gbs / peak) if pre_gbs else None, "peak_source": f"{peak_kind} hbm_gbs",
                "traffic": traffic,
                "algorithmic_bytes": pt.pre_levels_bytes}
    eval_bytes = pt.post_levels_bytes + pt.fused_bytes + pt.pre_levels_bytes
    na = max(pt_all.evals, 1)
    phases = {"source": f"separate pass of {pt_all.evals} evaluations with an event at every phase "
                        "boundary (which ends the programmatic overlap there: the phases sum to more "
                        "than the timed region's evaluation)",
              "pmatrix_ms": pt_all.pmatrix_ms / na, "post_levels_ms": pt_all.post_levels_ms / na,
              "fused_ms": pt_all.fused_ms / na, "pre_levels_ms": pt_all.pre_levels_ms / na,
              "reduce_ms": pt_all.reduce_ms / na, "eval_ms": pt_all.total_ms / na,
              "timed_region_pre_levels_ms": pre_ms, "timed_region_eval_ms": ms_per_step,
              "eval_algorithmic_bytes": eval_bytes,
              "eval_frac_of_peak": eval_bytes / (ms_per_step * 1e-3) / 1e9 / peak if ms_per_step else None}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_tips": 1000, "n_patterns": int(info.n_patterns),
                   "n_categories": 4, "n_states": 4, "partials": "fp32",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: each evaluation streams ~3.4 GB of partials, 26x the 129 MB L2",
                   "status": status},
        "roofline": roofline,
        "phases": phases,
        "e2e": e2e,
        "gpu_launches": pt.launches_per_eval * args.steps,
        "clocks": clocks.summary(),
    }
    if rank == 0 and world == 1:
        line["cpu_baseline"], ref, sample = _cpu_baseline(pr)
        line["error"] = _stated_error(ctx, pr, ref, sample, local)
    h.close()
    ctx.close()
    if rank == 0 and not args.no_extras:
        line["small"] = _small(local)
        line["codon"] = _codon(local)
        line["differentiation"] = _differentiation(local)
        line["inference"] = _inference(local)
        line["hmc"] = _hmc(local)
        if args.serving_requests > 0:
            line["serving"] = _serving(args.serving_requests, local)
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=800)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("gpu", "reference"), default="gpu")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the serving measurement (0 skips it)")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline nucleotide measurement (no codon, differentiation, serving)")
    ap.add_argument("--case", choices=("all", "codon", "differentiation", "hmc", "small"), default="all",
                    help="codon / differentiation: time that workload alone for --steps steps after "
                         "--warmup (for profiling); hmc, small: that object alone; all: the full measurement")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    from paper_1905_12146_gb300 import build
    build.build()
    if args.case != "all":
        _, _, local = _rank_env()
        if args.case in ("hmc", "small"):
            fn = _hmc if args.case == "hmc" else _small
            print(json.dumps({"case": args.case, **fn(local)}), flush=True)
            return 0
        if args.case == "codon":
            out = _codon(local, steps=args.steps, warmup=args.warmup, error=False)
        else:
            out = _differentiation(local, steps=args.steps, warmup=args.warmup)
        print(json.dumps({"case": args.case, **out}), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
