"""The binding's ctypes structures against the C header's layout, on the CPU.

Every public struct of include/qmccpw.h is compiled with the host C compiler,
which prints its size and each field's offset; the ctypes mirror in
paper_2209_11337_gb300/qmccpw.py must agree field by field (same names, same
order, same offsets, same size), so no argument is marshalled into the wrong
bytes."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2209_11337_gb300 import qmccpw as q

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = ["qmccpw_plan_desc", "qmccpw_option", "qmccpw_market", "qmccpw_result", "qmccpw_contract",
           "qmccpw_server_desc", "qmccpw_server_stats", "qmccpw_basket", "qmccpw_pipe_peaks"]


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qmccpw.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'    printf("{s} . %zu\\n", sizeof({s}));')
        for name, _ in getattr(q, s)._fields_:
            lines.append(f'    printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    lines += ["    return 0;", "}"]
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.strip().splitlines():
        s, name, value = line.split()
        table[(s, name)] = int(value)
    return table


@pytest.mark.parametrize("struct", STRUCTS)
def test_ctypes_mirror_matches_the_header(layout, struct):
    cls = getattr(q, struct)
    assert ctypes.sizeof(cls) == layout[(struct, ".")], struct
    for name, _ in cls._fields_:
        assert getattr(cls, name).offset == layout[(struct, name)], (struct, name)
