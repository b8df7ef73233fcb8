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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: size and every field offset,
    printed by a C program compiled against include/phylograd.h."""
    import subprocess

    from paper_1905_12146_gb300 import _native
    structs = {"pg_problem": _native.pg_problem, "pg_options": _native.pg_options,
               "pg_server_options": _native.pg_server_options, "pg_request": _native.pg_request,
               "pg_request_info": _native.pg_request_info, "pg_handle_info": _native.pg_handle_info,
               "pg_phase_times": _native.pg_phase_times}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "phylograd.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[f"{name} size"]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name} {field}"]) == getattr(cls, field).offset, (name, field)


def test_binding_marshals_tip_partials():
    import numpy as np

    from paper_1905_12146_gb300 import _native
    from paper_1905_12146_gb300 import workloads as wl
    pr = wl.random_problem(6, 20, seed=3)
    st, _ = _native.problem_struct(pr)
    assert st.n_tip_partials == 0 and not st.tip_partials
    table = wl.iupac_nucleotide_partials()
    pr = dict(pr, tip_partials=table,
              tip_states=wl.make_partially_observed(pr["tip_states"], 0.3, table, np.random.default_rng(0)))
    with pytest.raises(ValueError):   # rows must have one entry per state
        _native.problem_struct(dict(pr, tip_partials=table[:, :3]))
    st, keep = _native.problem_struct(pr)
    assert st.n_tip_partials == table.shape[0]
    buf = (ctypes.c_double * table.size).from_address(st.tip_partials)
    np.testing.assert_array_equal(np.frombuffer(buf, dtype=np.float64).reshape(table.shape), table)
