"""The Python binding's ctypes mirrors of the C-ABI structs match include/mcrt.h.

A small C program, compiled here with the host compiler against the header,
prints each struct's size and every field's offset; the ctypes classes of
paper_1810_00188_gb300/mcrt.py must agree field by field and in order, so a
field added to the header (or moved) without its mirror fails here rather than
corrupting a call.  No GPU is needed.
"""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_1810_00188_gb300 import mcrt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["mcrt_grid_desc", "mcrt_kdist_desc", "mcrt_solve_params", "mcrt_solve_stats",
           "mcrt_tuning", "mcrt_batch_item"]


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mcrt.h"', "int main(void) {"]
    for name in STRUCTS:
        cls = getattr(mcrt, name)
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr  # a mirrored field missing from the header fails to compile
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


def _header_fields(name):
    """Field names of a typedef'd struct of the header, in order (comments removed)."""
    src = open(os.path.join(ROOT, "include", "mcrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    m = re.search(r"typedef\s+struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        # "const double *nu_c, *dnu" / "int box[6]" / "double eps_wall[2]"
        names = [decl.split()[-1]]
        if "," in decl:
            first = decl.split(",")[0].split()[-1]
            names = [first] + [p.strip() for p in decl.split(",")[1:]]
        for nm in names:
            fields.append(re.sub(r"\[.*\]", "", nm).lstrip("*").strip())
    return fields


@pytest.mark.parametrize("name", STRUCTS)
def test_ctypes_mirror_has_the_header_fields_in_order(name):
    cls = getattr(mcrt, name)
    assert [f for f, _ in cls._fields_] == _header_fields(name)


def test_ctypes_offsets_and_sizes_match_the_c_compiler(tmp_path):
    layout = _c_layout(tmp_path)
    for name in STRUCTS:
        cls = getattr(mcrt, name)
        assert C.sizeof(cls) == layout[(name, "size")], name
        for field, _ in cls._fields_:
            assert getattr(cls, field).offset == layout[(name, field)], (name, field)
