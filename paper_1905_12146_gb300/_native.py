"""Thin ctypes binding of libphylograd.so (argument marshalling only).

Every computation happens in the CUDA library; this module converts numpy arrays and torch
device tensors into the pointers and sizes of the C ABI in ``include/phylograd.h`` and turns
status codes into exceptions.  If the library has not been built, importing works but the first
call raises ``RuntimeError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libphylograd.so")

PRECISIONS = {"fp32": 0, "fp64": 1}
PG_OK, PG_ERR_INVALID, PG_ERR_OOM, PG_ERR_CUDA, PG_ERR_TIMEOUT, PG_ERR_NUMERIC, PG_ERR_UNSUPPORTED = range(7)

EXPORTED = ("pg_create", "pg_destroy", "pg_upload", "pg_free", "pg_eval", "pg_eval_async",
            "pg_eval_batch_async", "pg_eval_status", "pg_get_info", "pg_set_phase_timing",
            "pg_get_phase_times", "pg_eval_noalloc", "pg_status_string", "pg_last_error",
            "pg_forward_async", "pg_backward_async", "pg_forward_batch_async",
            "pg_backward_batch_async", "pg_clock_lengths_async", "pg_clock_grad_async",
            "pg_server_create", "pg_server_submit", "pg_server_wait", "pg_server_destroy",
            "pg_selftest_timeout")


class PhyloGradError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


class pg_options(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("patterns_per_tile", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_uint64), ("flags", ctypes.c_uint32)]


PG_FLAG_SIMT_MSTATE = 1
PG_FLAG_FP64_DEVICE_PARTIALS = 2


class pg_problem(ctypes.Structure):
    _fields_ = [("n_tips", ctypes.c_int32), ("n_states", ctypes.c_int32),
                ("n_patterns", ctypes.c_int32), ("n_categories", ctypes.c_int32),
                ("n_models", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("parent", ctypes.c_void_p), ("tip_states", ctypes.c_void_p),
                ("pattern_weights", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("branch_model", ctypes.c_void_p), ("root_freqs", ctypes.c_void_p),
                ("cat_rates", ctypes.c_void_p), ("cat_weights", ctypes.c_void_p),
                ("tip_stride", ctypes.c_int32), ("n_tip_partials", ctypes.c_int32),
                ("tip_partials", ctypes.c_void_p), ("n_nodes", ctypes.c_int32)]


class pg_server_options(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("arena_bytes", ctypes.c_uint64)]


class pg_request(ctypes.Structure):
    _fields_ = [("problem", ctypes.c_void_p), ("b", ctypes.c_void_p), ("logL", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("hess", ctypes.c_void_p)]


class pg_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_int32), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class pg_handle_info(ctypes.Structure):
    _fields_ = [("n_tips", ctypes.c_int32), ("n_nodes", ctypes.c_int32),
                ("n_states", ctypes.c_int32), ("n_patterns", ctypes.c_int32),
                ("n_categories", ctypes.c_int32), ("n_levels", ctypes.c_int32),
                ("n_tiles", ctypes.c_int32), ("patterns_per_tile", ctypes.c_int32),
                ("device_bytes", ctypes.c_uint64), ("stream_bytes", ctypes.c_uint64),
                ("flops", ctypes.c_uint64)]


class pg_phase_times(ctypes.Structure):
    _fields_ = [("pmatrix_ms", ctypes.c_double), ("post_levels_ms", ctypes.c_double),
                ("fused_ms", ctypes.c_double), ("pre_levels_ms", ctypes.c_double),
                ("reduce_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("evals", ctypes.c_int32), ("launches_per_eval", ctypes.c_int32),
                ("post_levels_bytes", ctypes.c_uint64), ("fused_bytes", ctypes.c_uint64),
                ("pre_levels_bytes", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it is missing: build it with ``build()`` first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -m paper_1905_12146_gb300.build)")
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    sig = {
        "pg_create": ([ctypes.POINTER(pg_options), ctypes.POINTER(vp)], i32),
        "pg_destroy": ([vp], i32),
        "pg_upload": ([vp, ctypes.POINTER(pg_problem), ctypes.POINTER(vp)], i32),
        "pg_free": ([vp], i32),
        "pg_eval": ([vp, vp, vp, vp, vp, vp], i32),
        "pg_eval_async": ([vp, vp, vp, vp, vp, vp, vp], i32),
        "pg_eval_batch_async": ([vp, i32, vp, vp, vp, vp, vp], i32),
        "pg_eval_status": ([vp], i32),
        "pg_get_info": ([vp, ctypes.POINTER(pg_handle_info)], i32),
        "pg_set_phase_timing": ([vp, i32], i32),
        "pg_get_phase_times": ([vp, ctypes.POINTER(pg_phase_times)], i32),
        "pg_eval_noalloc": ([ctypes.POINTER(pg_problem), vp, vp, vp, vp, vp, vp], i32),
        "pg_forward_async": ([vp, vp, vp, vp, vp], i32),
        "pg_backward_async": ([vp, vp, vp, vp, vp], i32),
        "pg_forward_batch_async": ([vp, i32, vp, vp, vp], i32),
        "pg_backward_batch_async": ([vp, i32, vp, vp, vp, vp], i32),
        "pg_clock_lengths_async": ([vp, i32, vp, vp, vp, vp, vp], i32),
        "pg_clock_grad_async": ([vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
        "pg_server_create": ([vp, ctypes.POINTER(pg_server_options), ctypes.POINTER(vp)], i32),
        "pg_server_submit": ([vp, ctypes.POINTER(pg_request), ctypes.POINTER(ctypes.c_uint64)], i32),
        "pg_server_wait": ([vp, ctypes.c_uint64, ctypes.POINTER(pg_request_info)], i32),
        "pg_server_destroy": ([vp], i32),
        "pg_selftest_timeout": ([vp, ctypes.c_uint64], i32),
        "pg_status_string": ([i32], ctypes.c_char_p),
        "pg_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(status: int):
    if status != PG_OK:
        lib = load()
        raise PhyloGradError(status, f"{lib.pg_status_string(status).decode()}: "
                                     f"{lib.pg_last_error().decode()}")


def _np_ptr(a):
    return None if a is None else a.ctypes.data


def _stream(stream):
    if stream is None:
        return None
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr_array(items):
    """A C array of device pointers (None entries become NULL); None for a missing list."""
    if items is None:
        return None
    arr = (ctypes.c_void_p * max(len(items), 1))(*[_dev_ptr(x) for x in items])
    return ctypes.cast(arr, ctypes.c_void_p), arr   # keep arr alive alongside the pointer


def _dev_ptr(t):
    """Device pointer of a torch CUDA tensor (or an int address, or None)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _tip_partials(problem: dict, m: int):
    """(K, [K][m] FP64 array or None) of the problem's optional tip partial vectors."""
    tv = problem.get("tip_partials")
    if tv is None or len(tv) == 0:
        return 0, None
    tv = np.ascontiguousarray(tv, dtype=np.float64)
    if tv.ndim != 2 or tv.shape[1] != m:
        raise ValueError(f"tip_partials must be [K][{m}]")
    return tv.shape[0], tv


def problem_struct(problem: dict, precision: str = "fp32"):
    """The pg_problem of a problem dict and the arrays it points into (keep both alive while the
    library may read them).  Tip rows may be a row-strided view (unit stride along patterns)."""
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    parent = np.ascontiguousarray(problem["parent"], dtype=np.int32)
    tips = np.asarray(problem["tip_states"])
    if tips.dtype != np.uint8 or tips.ndim != 2 or tips.strides[1] != 1 or tips.strides[0] < tips.shape[1]:
        tips = np.ascontiguousarray(tips, dtype=np.uint8)
    stride = int(tips.strides[0]) if tips.ndim == 2 and tips.shape[0] > 1 else 0
    w = np.ascontiguousarray(problem["weights"], dtype=np.float64)
    Q = np.ascontiguousarray(problem["Q"], dtype=np.float64)
    if Q.ndim == 2:
        Q = Q[None]
    bm = problem.get("branch_model")
    bm = None if bm is None else np.ascontiguousarray(bm, dtype=np.int32)
    pi = np.ascontiguousarray(problem["root_freqs"], dtype=np.float64)
    rates = np.ascontiguousarray(problem["cat_rates"], dtype=np.float64)
    cw = np.ascontiguousarray(problem["cat_weights"], dtype=np.float64)
    n = parent.shape[0]
    P = tips.shape[1] if tips.ndim == 2 else 0
    K, tv = _tip_partials(problem, Q.shape[1])
    pr = pg_problem(_n_tips(problem, n), Q.shape[1], P, rates.shape[0], Q.shape[0], PRECISIONS[precision],
                    _np_ptr(parent), _np_ptr(tips), _np_ptr(w), _np_ptr(Q), _np_ptr(bm), _np_ptr(pi),
                    _np_ptr(rates), _np_ptr(cw), stride if stride != P else 0, K, _np_ptr(tv), n)
    return pr, (parent, tips, w, Q, bm, pi, rates, cw, tv)


def _n_tips(problem: dict, n: int) -> int:
    """Tips of a problem with n nodes: problem["n_tips"], else those of a binary tree."""
    return int(problem.get("n_tips", (n + 1) // 2))


class Context:
    """One CUDA device with an optional device-memory budget (pg_create / pg_destroy)."""

    def __init__(self, device: int = 0, patterns_per_tile: int = 0, hbm_budget_bytes: int = 0, flags: int = 0):
        lib = load()
        opt = pg_options(device, patterns_per_tile, hbm_budget_bytes, flags)
        out = ctypes.c_void_p()
        check(lib.pg_create(ctypes.byref(opt), ctypes.byref(out)))
        self._ptr = out
        self.device = device

    def selftest_timeout(self, limit_cycles: int = 2_000_000) -> int:
        """Run the library's bounded device-side wait on a barrier nothing arrives at; returns the
        status (PG_ERR_TIMEOUT when the wait gave up as intended)."""
        return int(load().pg_selftest_timeout(self._ptr, int(limit_cycles)))

    def upload(self, problem: dict, precision: str | None = None) -> "Handle":
        """pg_upload of a problem dict: parent, tip_states [N][P] (uint8 codes), weights, Q
        ([models][m][m] or [m][m]), root_freqs, cat_rates, cat_weights; optional branch_model and
        tip_partials [K][m] (codes m .. m+K-1 select its rows, partially observed tips)."""
        return Handle(self, problem, precision)

    def close(self):
        if self._ptr:
            load().pg_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle:
    """A device-resident problem (pg_upload); evaluations via pg_eval / pg_eval_async."""

    def __init__(self, ctx: Context, problem: dict, precision: str | None = None):
        lib = load()
        precision = precision or problem.get("precision", "fp32")
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.ctx = ctx
        pr, _keep = problem_struct(problem, precision)
        n = pr.n_nodes
        self.root = int(np.flatnonzero(_keep[0] < 0)[0])
        out = ctypes.c_void_p()
        check(lib.pg_upload(ctx._ptr, ctypes.byref(pr), ctypes.byref(out)))
        self._ptr = out
        self.n_nodes = n
        self.n_patterns = pr.n_patterns

    def info(self) -> pg_handle_info:
        info = pg_handle_info()
        check(load().pg_get_info(self._ptr, ctypes.byref(info)))
        return info

    def eval(self, b, grad=True, hess=False, site=False):
        """Blocking evaluation with host arrays (pg_eval).  Returns a dict."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        if b.shape != (self.n_nodes,):
            raise ValueError(f"b must have shape ({self.n_nodes},)")
        logL = np.zeros(1)
        g = np.zeros(self.n_nodes) if grad else None
        h = np.zeros(self.n_nodes) if hess else None
        s = np.zeros(self.n_patterns) if site else None
        st = load().pg_eval(self._ptr, _np_ptr(b), _np_ptr(logL), _np_ptr(g), _np_ptr(h), _np_ptr(s))
        out = {"logL": float(logL[0]), "grad": g, "hess": h, "site_logL": s, "status": st}
        if st not in (PG_OK, PG_ERR_NUMERIC):
            check(st)
        return out

    def eval_async(self, d_b, d_logL, d_grad=None, d_hess=None, d_site=None, stream=None):
        """Enqueue an evaluation on ``stream`` (a torch.cuda.Stream, a raw handle or None) with
        device tensors/pointers."""
        s = None
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        check(load().pg_eval_async(self._ptr, _dev_ptr(d_b), _dev_ptr(d_logL), _dev_ptr(d_grad),
                                   _dev_ptr(d_hess), _dev_ptr(d_site), s))

    def forward_async(self, d_b, d_logL, d_site=None, stream=None):
        """pg_forward_async: P build, post-order and root (logL only); partials stay resident."""
        check(load().pg_forward_async(self._ptr, _dev_ptr(d_b), _dev_ptr(d_logL), _dev_ptr(d_site),
                                      _stream(stream)))

    def backward_async(self, d_gscale, d_grad, d_hess=None, stream=None):
        """pg_backward_async: pre-order pass and gradient (times *d_gscale) from the last forward."""
        check(load().pg_backward_async(self._ptr, _dev_ptr(d_gscale), _dev_ptr(d_grad), _dev_ptr(d_hess),
                                       _stream(stream)))

    def set_phase_timing(self, mode):
        """pg_set_phase_timing: False/0 off, True/1 every phase boundary, 2 the pre-order levels only,
        3 those of every 8th evaluation."""
        check(load().pg_set_phase_timing(self._ptr, int(mode)))

    def phase_times(self) -> pg_phase_times:
        out = pg_phase_times()
        check(load().pg_get_phase_times(self._ptr, ctypes.byref(out)))
        return out

    def status(self) -> int:
        return load().pg_eval_status(self._ptr)

    def close(self):
        if self._ptr:
            load().pg_free(self._ptr)
            self._ptr = None


def eval_batch_async(handles, d_b, d_logL, d_grad=None, d_hess=None, stream=None):
    """pg_eval_batch_async over a list of handles with per-problem device tensors."""
    k = len(handles)
    VP = ctypes.c_void_p * max(k, 1)
    hs = VP(*[h._ptr.value for h in handles])
    bs = VP(*[_dev_ptr(x) for x in d_b])
    gs = VP(*[_dev_ptr(x) for x in d_grad]) if d_grad is not None else None
    hh = VP(*[_dev_ptr(x) for x in d_hess]) if d_hess is not None else None
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    check(load().pg_eval_batch_async(ctypes.cast(hs, ctypes.c_void_p), k,
                                     ctypes.cast(bs, ctypes.c_void_p), _dev_ptr(d_logL),
                                     None if gs is None else ctypes.cast(gs, ctypes.c_void_p),
                                     None if hh is None else ctypes.cast(hh, ctypes.c_void_p), s))


def _handles(handles):
    k = len(handles)
    hs = (ctypes.c_void_p * max(k, 1))(*[h._ptr.value for h in handles])
    return k, ctypes.cast(hs, ctypes.c_void_p), hs


def _arg(pa):
    return None if pa is None else pa[0]


def forward_batch_async(handles, d_b, d_logL, stream=None):
    """pg_forward_batch_async: logL of every problem into the device array d_logL [k]."""
    k, hp, _keep = _handles(handles)
    bs = _ptr_array(d_b)
    check(load().pg_forward_batch_async(hp, k, _arg(bs), _dev_ptr(d_logL), _stream(stream)))


def backward_batch_async(handles, d_gscale, d_grad, d_hess=None, stream=None):
    """pg_backward_batch_async: gradient of problem i times d_gscale[i] into d_grad[i]."""
    k, hp, _keep = _handles(handles)
    gs, hh = _ptr_array(d_grad), _ptr_array(d_hess)
    check(load().pg_backward_batch_async(hp, k, _dev_ptr(d_gscale), _arg(gs), _arg(hh), _stream(stream)))


def clock_lengths_async(handles, d_eps, d_mu, d_t, d_b, stream=None):
    """pg_clock_lengths_async: b_i = mu eps_i (t_i - t_parent(i)) per problem."""
    k, hp, _keep = _handles(handles)
    e, t, b = _ptr_array(d_eps), _ptr_array(d_t), _ptr_array(d_b)
    check(load().pg_clock_lengths_async(hp, k, _arg(e), _dev_ptr(d_mu), _arg(t), _arg(b), _stream(stream)))


def clock_grad_async(handles, d_eps, d_mu, d_t, d_grad_b, d_grad_eps=None, d_grad_mu=None, d_grad_t=None,
                     d_grad_rate=None, stream=None):
    """pg_clock_grad_async: chain rule of dlogL/db to eps, mu, node times and rates."""
    k, hp, _keep = _handles(handles)
    e, t, g = _ptr_array(d_eps), _ptr_array(d_t), _ptr_array(d_grad_b)
    ge, gt, gr = _ptr_array(d_grad_eps), _ptr_array(d_grad_t), _ptr_array(d_grad_rate)
    check(load().pg_clock_grad_async(hp, k, _arg(e), _dev_ptr(d_mu), _arg(t), _arg(g), _arg(ge),
                                     _dev_ptr(d_grad_mu), _arg(gt), _arg(gr), _stream(stream)))


def eval_noalloc(problem: dict, b, precision: str = "fp32", grad=True, hess=False, site=False,
                 stream=None):
    """pg_eval_noalloc: one blocking evaluation with host arrays that allocates no device or host
    heap memory inside the library (its scratch is a fixed per-GPU device array).  For callers that
    cannot allocate at evaluation time; calls must not overlap.  Returns a dict like Handle.eval."""
    lib = load()
    parent = np.ascontiguousarray(problem["parent"], dtype=np.int32)
    tips = np.ascontiguousarray(problem["tip_states"], dtype=np.uint8)
    w = np.ascontiguousarray(problem["weights"], dtype=np.float64)
    Q = np.ascontiguousarray(problem["Q"], dtype=np.float64)
    if Q.ndim == 2:
        Q = Q[None]
    bm = problem.get("branch_model")
    bm = None if bm is None else np.ascontiguousarray(bm, dtype=np.int32)
    pi = np.ascontiguousarray(problem["root_freqs"], dtype=np.float64)
    rates = np.ascontiguousarray(problem["cat_rates"], dtype=np.float64)
    cw = np.ascontiguousarray(problem["cat_weights"], dtype=np.float64)
    n = parent.shape[0]
    P = tips.shape[1] if tips.ndim == 2 else 0
    K, tv = _tip_partials(problem, Q.shape[1])
    pr = pg_problem(_n_tips(problem, n), Q.shape[1], P, rates.shape[0], Q.shape[0], PRECISIONS[precision],
                    _np_ptr(parent), _np_ptr(tips), _np_ptr(w), _np_ptr(Q), _np_ptr(bm),
                    _np_ptr(pi), _np_ptr(rates), _np_ptr(cw), 0, K, _np_ptr(tv), n)
    b = np.ascontiguousarray(b, dtype=np.float64)
    logL = np.zeros(1)
    g = np.zeros(n) if grad else None
    h = np.zeros(n) if hess else None
    st_site = np.zeros(P) if site else None
    s = None
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib.pg_eval_noalloc(ctypes.byref(pr), _np_ptr(b), _np_ptr(logL), _np_ptr(g), _np_ptr(h),
                             _np_ptr(st_site), s)
    out = {"logL": float(logL[0]), "grad": g, "hess": h, "site_logL": st_site, "status": st}
    if st not in (PG_OK, PG_ERR_NUMERIC):
        check(st)
    return out


class Server:
    """Continuous-batching request server (pg_server_*): submit(problem, b) queues a request and
    returns a ticket; wait(ticket) blocks until it completes and returns its results and times."""

    def __init__(self, ctx: Context, max_inflight: int = 4, arena_bytes: int = 0):
        lib = load()
        opt = pg_server_options(max_inflight, 0, arena_bytes)
        out = ctypes.c_void_p()
        check(lib.pg_server_create(ctx._ptr, ctypes.byref(opt), ctypes.byref(out)))
        self._ptr = out
        self.ctx = ctx
        self._live = {}

    def submit(self, problem: dict, b=None, grad=True, hess=False) -> int:
        pr, keep = problem_struct(problem, problem.get("precision", "fp32"))
        n = pr.n_nodes
        b = np.ascontiguousarray(problem["b"] if b is None else b, dtype=np.float64)
        if b.shape != (n,):
            raise ValueError(f"b must have shape ({n},)")
        out = {"logL": np.zeros(1), "grad": np.zeros(n) if grad else None, "hess": np.zeros(n) if hess else None}
        rq = pg_request(ctypes.addressof(pr), _np_ptr(b), _np_ptr(out["logL"]), _np_ptr(out["grad"]),
                        _np_ptr(out["hess"]))
        ticket = ctypes.c_uint64()
        check(load().pg_server_submit(self._ptr, ctypes.byref(rq), ctypes.byref(ticket)))
        self._live[ticket.value] = (pr, keep, b, out, rq)
        return ticket.value

    def wait(self, ticket: int) -> dict:
        info = pg_request_info()
        st = load().pg_server_wait(self._ptr, ticket, ctypes.byref(info))
        pr, keep, b, out, rq = self._live.pop(ticket)
        if st not in (PG_OK, PG_ERR_NUMERIC):
            check(st)
        return {"logL": float(out["logL"][0]), "grad": out["grad"], "hess": out["hess"], "status": st,
                "submit_s": info.submit_s, "start_s": info.start_s, "done_s": info.done_s}

    def close(self):
        if self._ptr:
            load().pg_server_destroy(self._ptr)
            self._ptr = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
