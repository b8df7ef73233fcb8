"""CPU checks of the boundary: the library builds for sm_103a, loads, and exports every function
declared in include/*.h (no compute call is made, so no GPU is needed)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(pg_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1905_12146_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    assert {"pg_create", "pg_upload", "pg_eval", "pg_eval_async", "pg_eval_batch_async",
            "pg_free", "pg_destroy", "pg_status_string"} <= names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1905_12146_gb300 import _native
    assert _declared() <= set(_native.EXPORTED)


def test_status_strings_are_host_only(lib_path):
    from paper_1905_12146_gb300 import _native
    lib = _native.load(lib_path)
    for code in range(7):
        assert lib.pg_status_string(code)
    assert lib.pg_status_string(99) == b"unknown status"



def test_selftest_rejects_a_null_context(lib_path):
    """Argument checks come before any CUDA call, so this runs without a GPU."""
    lib = ctypes.CDLL(lib_path)
    lib.pg_selftest_timeout.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    lib.pg_selftest_timeout.restype = ctypes.c_int32
    assert lib.pg_selftest_timeout(None, 1_000_000) == 1   # PG_ERR_INVALID


def test_binding_refuses_partially_observed_tips():
    """Tip-partial tables are an oracle-only input for now: the binding refuses them rather than
    letting the library read their codes as missing data."""
    import numpy as np

    from paper_1905_12146_gb300 import _native
    from paper_1905_12146_gb300 import workloads as wl
    pr = wl.random_problem(6, 20, seed=3)
    _native.problem_struct(pr)   # plain codes marshal
    table = wl.iupac_nucleotide_partials()
    pr = dict(pr, tip_partials=table,
              tip_states=wl.make_partially_observed(pr["tip_states"], 0.3, table, np.random.default_rng(0)))
    with pytest.raises(NotImplementedError):
        _native.problem_struct(pr)
    with pytest.raises(NotImplementedError):
        _native.eval_noalloc(pr, pr["b"])
