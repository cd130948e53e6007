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


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the C header's sizes and field
    offsets (a field added on one side only would pass garbage across the ABI)."""
    import shutil
    import subprocess

    import pytest

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1607_02573_gb300 import mwi
    structs = {"mwi_solver_opts": mwi.mwi_solver_opts, "mwi_solve_info": mwi.mwi_solve_info,
               "mwi_antenna": mwi.mwi_antenna}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mwi.h"', "int main(void) {"]
    for name, st in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        name, what, val = line.split()
        st = structs[name]
        want = ctypes.sizeof(st) if what == "size" else getattr(st, what).offset
        assert int(val) == want, (name, what, int(val), want)
