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
