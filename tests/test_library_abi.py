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


def test_mesh_create_rejects_bad_meshes_on_the_host():
    """Mesh validation happens on the host before any device work: a degenerate
    or vertex-repeating tet, an out-of-range vertex id and a bad boundary tag
    each give MWI_EINVAL with a message (no GPU needed)."""
    import numpy as np

    from paper_1607_02573_gb300 import mwi
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0]], dtype=np.float64)
    good = np.array([[0, 1, 2, 3]], dtype=np.int32)
    tag = np.zeros((1, 4), dtype=np.int32)
    cases = {
        "degenerate": (np.array([[0, 1, 2, 4]], dtype=np.int32), tag),  # four coplanar vertices
        "repeat": (np.array([[0, 1, 1, 3]], dtype=np.int32), tag),
        "range": (np.array([[0, 1, 2, 7]], dtype=np.int32), tag),
        "tag": (good, np.array([[0, 3, 0, 0]], dtype=np.int32)),
    }
    for name, (tet, tg) in cases.items():
        h = ctypes.c_void_p()
        st = mwi.mwi_mesh_create(mwi._ptr(xyz, ctypes.c_double), xyz.shape[0], mwi._ptr(tet, ctypes.c_int32), 1,
                                 mwi._ptr(tg, ctypes.c_int32), 1, ctypes.byref(h))
        assert st == mwi.MWI_EINVAL, name
        assert mwi.mwi_last_error(), name
        assert not h.value, name
