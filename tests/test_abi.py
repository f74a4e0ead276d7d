"""The C ABI library loads and exports every function include/*.h declares
(no compute call: runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        src = re.sub(r"^\s*#[^\n]*", "", src, flags=re.M)     # preprocessor lines
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(([^;{]*?)\)\s*;", src):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2510_25938_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))
    return ctypes.CDLL(path)


def test_header_declares_the_three_entry_points():
    names = declared_functions()
    for n in ("lj_energy_grad_batched", "lbfgs_minimize_batched", "bh_step_batched",
              "lj_ctx_create", "lj_ctx_destroy", "lj_ctx_reserve", "lj_status_string",
              "lj_ctx_last_error"):
        assert n in names


def test_library_exports_every_declared_function(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_status_strings_without_gpu(lib):
    lib.lj_status_string.restype = ctypes.c_char_p
    assert lib.lj_status_string(0) == b"LJ_OK"
    assert lib.lj_status_string(-4) == b"LJ_ERR_UNSUPPORTED"


def test_binding_names_match_abi():
    from paper_2510_25938_gb300 import lj_bh
    for n in ("lj_energy_grad_batched", "lbfgs_minimize_batched", "bh_step_batched"):
        assert callable(getattr(lj_bh, n))


def test_null_ctx_is_rejected(lib):
    lib.lbfgs_minimize_batched.restype = ctypes.c_int
    assert lib.lbfgs_minimize_batched(None, None, None, None, None, None, None, None, None,
                                      None) == -1
    lib.lj_ctx_get_tuning.restype = ctypes.c_int
    assert lib.lj_ctx_get_tuning(None, 0, None) == -1
    lib.lj_ctx_autotune_bh.restype = ctypes.c_int
    assert lib.lj_ctx_autotune_bh(None, None, None, None, None) == -1
    lib.lj_energy_grad_batched_pot.restype = ctypes.c_int
    assert lib.lj_energy_grad_batched_pot(None, None, 0, 0, None, None, None, 1,
                                          ctypes.c_double(1.0), ctypes.c_double(1.0),
                                          ctypes.c_double(6.0), None) == -1


def test_binding_struct_layouts_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the C struct's size and field
    offsets (a C program built against include/lj_bh.h prints them)."""
    import subprocess
    from paper_2510_25938_gb300 import lj_bh as L
    pairs = {"lj_batch": L._Batch, "lj_lbfgs_params": L._Lbfgs, "lj_bh_params": L._Bh,
             "lj_bh_state": L._State, "lj_bh_trace": L._Trace, "lj_tuning": L._Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lj_bh.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, val = line.split()
        got[(name, field)] = int(val)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
