"""The Python binding against the C header, on the CPU: every constant the binding
mirrors (precisions, flags, kernel ids) has the header's value, and every ctypes
structure has the header struct's field offsets and size (a plain C program compiled
with gcc prints them)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2509_11152_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "h2rs.h")


def _header_constants():
    text = open(HEADER).read()
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(H2_\w+)\s+(-?\d+)\b", text)}
    for m in re.finditer(r"\b(H2_(?:PREC|K|ERR)_\w+)\s*=\s*(-?\d+)", text):
        vals[m.group(1)] = int(m.group(2))
    return vals


def test_binding_constants_match_the_header():
    h = _header_constants()
    mirrored = {k: v for k, v in vars(B).items() if re.fullmatch(r"H2_(PREC|FLAG)_\w+", k)}
    assert mirrored, "the binding mirrors no constants"
    for k, v in mirrored.items():
        assert k in h and h[k] == v, (k, v, h.get(k))
    # every flag of the header is available from Python
    for k in h:
        if k.startswith("H2_FLAG_"):
            assert getattr(B, k) == h[k], k
    # kernel-id names in the header's order
    ids = sorted((v, k) for k, v in h.items() if k.startswith("H2_K_") and k != "H2_K_COUNT")
    assert [k[len("H2_K_"):].lower() for _, k in ids] == B.KERNELS
    assert h["H2_K_COUNT"] == len(B.KERNELS)
    assert len(B.PHASES) == 8


STRUCTS = {"h2_matrix_desc": B.h2_matrix_desc, "h2_factor_opts": B.h2_factor_opts,
           "h2_factor_stats": B.h2_factor_stats}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_ctypes_structs_match_the_header_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "h2rs.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (l.split() for l in out if l.strip())}
    for cname, cls in STRUCTS.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
