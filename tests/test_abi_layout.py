"""The ctypes structures of the binding match the C header's layouts.

A small C program compiled against include/tsbts.h prints the size of
each public struct and the offset of each field; the ctypes Structures in
paper_1205_2288_gb300/tsbts.py must agree field by field (a mismatch would
silently mix up configuration or statistics fields).
"""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1205_2288_gb300 import tsbts

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "tsbts_config": tsbts.tsbts_config,
    "tsbts_stats": tsbts.tsbts_stats,
    "tsbts_adjoint_stats": tsbts.tsbts_adjoint_stats,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>',
             '#include "tsbts.h"', 'int main(void) {']
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", '
                         f'offsetof({name}, {field}));')
    lines += ['  return 0;', '}']
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True,
                         text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, field, value = line.split()
        layout[(name, field)] = int(value)
    return layout


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_struct_layout_matches_header(c_layout, name):
    cls = STRUCTS[name]
    assert C.sizeof(cls) == c_layout[(name, "sizeof")]
    for field, _ in cls._fields_:
        assert getattr(cls, field).offset == c_layout[(name, field)], field
