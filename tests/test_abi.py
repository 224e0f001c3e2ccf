"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/mlev.h declares. No compute calls (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mlev.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mlev_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    from paper_1401_4969_gb300 import mlev

    lib = mlev.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(mlev.EXPORTS) == names


def test_struct_layouts_match_header():
    from paper_1401_4969_gb300 import mlev

    assert C.sizeof(mlev.Opts) == 80
    assert mlev.Opts.level1_tol.offset == 32
    assert mlev.Report.lambda_.offset == 8
