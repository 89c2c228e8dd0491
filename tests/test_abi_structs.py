"""The ctypes structures of the binding match the C structs of include/fast.h
field for field: names, order, types, offsets and sizes (CPU only; the
offsets come from a small C program compiled against the header)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fast.h")
STRUCTS = ("fast_params", "fast_stats", "fast_plan_choice", "fast_plan_info_t")


def header_structs():
    """{struct name: [(field, c type, array length or 0)]} for the typedef'd structs."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(\w+)\s*;", text, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            ctype, names = decl.split(None, 1)
            for n in names.split(","):
                n = n.strip()
                m = re.fullmatch(r"(\w+)\[(\d+)\]", n)
                fields.append((m.group(1), ctype, int(m.group(2))) if m else (n, ctype, 0))
        out[name] = fields
    return out


def ctypes_struct(name):
    from paper_1803_09835_gb300 import _lib
    return getattr(_lib, name)


CTYPE = {"uint32_t": ctypes.c_uint32, "uint64_t": ctypes.c_uint64, "float": ctypes.c_float}


@pytest.mark.parametrize("name", STRUCTS)
def test_fields_match_the_header(name):
    hdr = header_structs()[name]
    cls = ctypes_struct(name)
    assert [f for f, _, _ in hdr] == [f for f, _ in cls._fields_]
    for (f, ctype, n), (_, pytype) in zip(hdr, cls._fields_):
        want = CTYPE.get(ctype) or ctypes_struct(ctype)
        if n:
            want = want * n
        assert pytype == want, f"{name}.{f}: {ctype}[{n}] vs {pytype}"


def test_offsets_and_sizes_match_the_compiler(tmp_path):
    hdr = header_structs()
    lines = ["#include <stddef.h>", "#include <stdio.h>", f'#include "{HEADER}"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} sizeof %zu\\n", sizeof({s}));')
        for f, _, _ in hdr[s]:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.check_call(["gcc", "-std=c11", "-o", str(exe), str(src)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for s in STRUCTS:
        cls = ctypes_struct(s)
        assert ctypes.sizeof(cls) == got[(s, "sizeof")], s
        for f, _ in cls._fields_:
            assert getattr(cls, f).offset == got[(s, f)], f"{s}.{f}"
