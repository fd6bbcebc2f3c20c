"""The ctypes structures of the Python binding have the layout of the C header:
the same field names in the same order, and the same size and field offsets as
gcc gives for include/agg.h on this host (no GPU needed).

A field renamed, inserted or retyped on one side only would otherwise pass
every CPU test and surface as a wrong value on the GPU.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agg.h")


def header_structs(path=HEADER):
    """{struct name: [field names in order]} for every struct the header defines."""
    text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"typedef\s+struct\s+(\w+)\s*\{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in m.group(2).split(";"):
            decl = decl.strip()
            for d in decl.split(",") if decl else []:  # "uint64_t a, b;" declares a and b
                fields.append(re.match(r".*?(\w+)\s*(\[[^\]]*\])?$", d.strip(), flags=re.S).group(1))
        out[m.group(3)] = fields
    return out


def binding_structs():
    from paper_1311_0059_gb300 import _abi
    return {n: getattr(_abi, n) for n in header_structs()
            if isinstance(getattr(_abi, n, None), type) and issubclass(getattr(_abi, n), ctypes.Structure)}


def test_every_header_struct_has_a_binding():
    missing = sorted(set(header_structs()) - set(binding_structs()))
    assert not missing, f"structs of agg.h without a ctypes binding: {missing}"


@pytest.mark.parametrize("name", sorted(header_structs()))
def test_field_names_and_order(name):
    cls = binding_structs()[name]
    assert [f for f, *_ in cls._fields_] == header_structs()[name]


def test_sizes_and_offsets_match_gcc(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = binding_structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "agg.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, *_ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), f"sizeof({name})"
        for f, *_ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, f"offsetof({name}, {f})"
