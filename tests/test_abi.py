"""Host-side checks of the C ABI boundary (no GPU needed).

* the library builds for sm_103a and exports every entry point that
  include/lqdd.h declares, and the ctypes binding wraps each under the same name;
* the ctypes structures have the size and field offsets of the C structures
  (checked by compiling a probe against the header with gcc);
* the product package never imports the oracle (no CPU fallback exists).
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lqdd.h")
PKG = os.path.join(ROOT, "paper_2407_08092_gb300")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lq_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2407_08092_gb300 import build
    return build.build()


def test_header_declares_the_expected_entry_points():
    names = declared_functions()
    for n in ("lq_create", "lq_destroy", "lq_set_gauge", "lq_apply", "lq_prepare", "lq_reconstruct",
              "lq_estimate_norm", "lq_smooth", "lq_solve", "lq_status_string", "lq_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lq_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and nothing else with the lq_ prefix leaks out
    assert exported == set(declared_functions())


def test_binding_names_match_header(lib_path):
    from paper_2407_08092_gb300 import lqdd
    for n in declared_functions():
        assert callable(getattr(lqdd, n)), n
        assert hasattr(lqdd.library(), n)


def test_kernel_class_names(lib_path):
    from paper_2407_08092_gb300 import lqdd
    names = [lqdd.lq_kernel_class_name(c) for c in range(lqdd.LQ_K_COUNT)]
    assert all(names) and len(set(names)) == len(names)
    assert lqdd.lq_kernel_class_name(lqdd.LQ_K_COUNT) == ""
    header = open(os.path.join(ROOT, "include", "lqdd.h")).read()
    enum = header[header.index("LQ_K_HOP_K1_F64 = 0"):header.index("LQ_K_COUNT")]
    assert len(re.findall(r"LQ_K_[A-Z0-9_]+", enum)) == lqdd.LQ_K_COUNT


def test_struct_layouts_match_header(tmp_path):
    from paper_2407_08092_gb300 import lqdd
    probe = tmp_path / "probe.c"
    structs = {"lq_lattice": lqdd.lq_lattice, "lq_solver_params": lqdd.lq_solver_params,
               "lq_stats": lqdd.lq_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lqdd.h"', 'int main(void){']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0;}")
    probe.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(probe), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_product_never_touches_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), fn
                assert "liboracle" not in text, fn


def test_unchecked_build_reports_no_index_checks(lib_path):
    """lq_bounds_check in the normal build touches no device: checked = 0 and LQ_OK."""
    from paper_2407_08092_gb300 import lqdd
    status, checked, violations, first = lqdd.lq_bounds_check()
    assert (status, checked, violations, first) == (lqdd.LQ_OK, 0, 0, 0)


def test_checked_build_exports_the_same_symbols(lib_path):
    """The index-checked build (-DLQ_BOUNDS) compiles and exports the same C ABI."""
    from paper_2407_08092_gb300 import build
    checked = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", checked], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lq_[a-z0-9_]+)$", out, flags=re.M))
    assert exported == set(declared_functions())
