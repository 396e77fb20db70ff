"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads, and
exports every function include/sfcdd.h declares (no compute calls without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2110_11211_gb300 import _lib
from paper_2110_11211_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "sfcdd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sfcdd_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    return build()


def test_header_and_binding_agree():
    assert header_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (sfcdd_\w+)", out))
    missing = [f for f in header_functions() if f not in exported]
    assert not missing, missing


def test_library_loads_and_reports_status_strings(libpath):
    L = _lib.lib()
    assert L.sfcdd_status_string(0) == b"ok"
    assert b"argument" in L.sfcdd_status_string(-1)
    opt = _lib.Options()
    L.sfcdd_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.weighting == 1 and opt.variant == 0 and opt.flexible == -1


def test_struct_layouts_match_the_header(tmp_path):
    """Every option, statistics, info and tuning struct of include/sfcdd.h has
    the size and field offsets of its ctypes mirror (a plain C program built
    against the header prints them)."""
    mirrors = {"sfcdd_options": _lib.Options, "sfcdd_stats": _lib.Stats,
               "sfcdd_info": _lib.Info, "sfcdd_tuning": _lib.Tuning}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "sfcdd.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, key, val = line.split()
            got[(cname, key)] = int(val)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert got[(cname, field)] == getattr(py, field).offset, (cname, field)
