"""The ctypes mirrors of the C-ABI structs match include/stokes.h.

A small C program, compiled here with the host compiler against the header,
prints sizeof and offsetof of every struct and field the Python binding
declares; each must equal the ctypes layout.  Catches a field added to the
header but not to the binding (or in another order), which would otherwise
pass silently and corrupt the arguments of every call.
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1406_6573_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["stokes_field", "stokes_mesh_desc", "stokes_params", "stokes_sizes", "stokes_kernel_time",
           "stokes_profile", "stokes_solver_opts", "stokes_solve_report"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "stokes.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(capi, name)
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    # the header only needs cudaStream_t-free declarations (streams are void*)
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    return got


def test_ctypes_structs_match_the_header(tmp_path):
    got = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(capi, name)
        assert C.sizeof(cls) == got[(name, "sizeof")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == got[(name, field)], (name, field)
