"""The C-ABI library loads and exports every entry point declared in include/mwi.h
(no compute calls: runs without a GPU)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mwi_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mwi_mesh_create", "mwi_assemble", "mwi_forward_solve", "mwi_misfit_and_gradient",
              "mwi_fields_device", "mwi_problem_destroy", "mwi_mesh_destroy", "mwi_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1607_02573_gb300 import build as b
    lib_path = b.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1607_02573_gb300 import mwi
    assert sorted(mwi.EXPORTED) == _declared()


def test_last_error_is_callable_without_gpu():
    from paper_1607_02573_gb300 import mwi
    assert isinstance(mwi.mwi_last_error(), bytes)
