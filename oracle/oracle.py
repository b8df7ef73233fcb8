"""ctypes front-end of the FP64 CPU oracle (``phylo_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg, never by the library.  It shares no code with the CUDA path.

``build()`` compiles the C file with plain gcc (no fused multiply-add contraction, so results
are the same on x86 and Arm); ``evaluate(problem, b)`` runs the whole method of the paper
(Sections 2.2-2.6) and returns logL, the branch gradient, per-site logL and the Hessian diagonal.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "phylo_oracle.c")
_LIB = os.path.join(_HERE, "libphylo_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        up = ctypes.POINTER(ctypes.c_uint8)
        lib.orc_expm.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_expm.restype = ctypes.c_int
        lib.orc_eval_tree.argtypes = [ctypes.c_int] * 6 + [ip, up, dp, dp, ip, dp, dp, dp, dp,
                                                           ctypes.c_int, dp,
                                                           dp, dp, dp, dp, dp, dp, ip, ip]
        lib.orc_eval_tree.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def expm(A: np.ndarray) -> np.ndarray:
    """e^A by the oracle's Pade scaling-and-squaring."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.empty_like(A)
    rc = _load().orc_expm(A.shape[0], _ptr(A, ctypes.c_double), _ptr(out, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"orc_expm failed ({rc})")
    return out


class OracleResult(dict):
    __getattr__ = dict.__getitem__


def evaluate(problem: dict, b: np.ndarray | None = None, partials: bool = False,
             patterns: slice | None = None) -> OracleResult:
    """Run the oracle on ``problem`` (a dict from ``workloads``) at branch lengths ``b``.

    The tree has ``problem["n_tips"]`` tips (nodes 0..N-1) and ``len(parent)`` nodes: 2N-1 for a
    binary tree, fewer when some internal nodes have more than two children.

    An optional ``problem["tip_partials"]`` [K][m] holds the partial vectors of partially observed
    tips: code m + k selects row k, codes from m + K on are missing data (all ones).

    ``patterns`` restricts the evaluation to a slice of the site patterns (the result is then the
    log-likelihood of that sub-alignment).  With ``partials=True`` the scaled post- and pre-order
    partials of every node are returned as ``post[n][P][C][m]``, ``pre[...]`` with their log2
    factors ``post_e[n][P]``, ``pre_e[n][P]``."""
    lib = _load()
    parent = np.ascontiguousarray(problem["parent"], dtype=np.int32)
    tips = problem["tip_states"]
    w = problem["weights"]
    if patterns is not None:
        tips = tips[:, patterns]
        w = w[patterns]
    tips = np.ascontiguousarray(tips, dtype=np.uint8)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Q = np.ascontiguousarray(problem["Q"], dtype=np.float64)
    if Q.ndim == 2:
        Q = Q[None]
    bm = problem.get("branch_model")
    bm = None if bm is None else np.ascontiguousarray(bm, dtype=np.int32)
    pi = np.ascontiguousarray(problem["root_freqs"], dtype=np.float64)
    rates = np.ascontiguousarray(problem["cat_rates"], dtype=np.float64)
    cw = np.ascontiguousarray(problem["cat_weights"], dtype=np.float64)
    b = np.ascontiguousarray(problem["b"] if b is None else b, dtype=np.float64)
    tv = problem.get("tip_partials")
    tv = None if tv is None or len(tv) == 0 else np.ascontiguousarray(tv, dtype=np.float64)
    n = parent.shape[0]
    n_tips = int(problem.get("n_tips", (n + 1) // 2))   # fewer than n = 2N-1 nodes: multifurcations
    m = Q.shape[1]
    if tv is not None and (tv.ndim != 2 or tv.shape[1] != m):
        raise ValueError("tip_partials must be [K][m]")
    P = tips.shape[1]
    C = rates.shape[0]
    logL = np.zeros(1)
    grad = np.zeros(n)
    hess = np.zeros(n)
    site = np.zeros(max(P, 1))
    post = pre = pe = qe = None
    if partials:
        post = np.zeros((n, P, C, m))
        pre = np.zeros((n, P, C, m))
        pe = np.zeros((n, P), dtype=np.int32)
        qe = np.zeros((n, P), dtype=np.int32)
    dp = ctypes.c_double
    rc = lib.orc_eval_tree(n_tips, n, m, P, C, Q.shape[0], _ptr(parent, ctypes.c_int32),
                      _ptr(tips, ctypes.c_uint8), _ptr(w, dp), _ptr(Q, dp),
                      _ptr(bm, ctypes.c_int32), _ptr(pi, dp), _ptr(rates, dp), _ptr(cw, dp),
                      _ptr(b, dp), 0 if tv is None else tv.shape[0], _ptr(tv, dp),
                      _ptr(logL, dp), _ptr(grad, dp), _ptr(site, dp), _ptr(hess, dp), _ptr(post, dp), _ptr(pre, dp),
                      _ptr(pe, ctypes.c_int32), _ptr(qe, ctypes.c_int32))
    if rc != 0:
        raise ValueError(f"orc_eval rejected the problem (code {rc})")
    out = OracleResult(logL=float(logL[0]), grad=grad, hess=hess, site_logL=site[:P])
    if partials:
        out.update(post=post, pre=pre, post_e=pe, pre_e=qe)
    return out
