"""The Python binding's ctypes structures against the C header: a small C
program built with the host compiler from include/pyhst.h prints sizeof and
every field's offsetof, and each must equal what ctypes lays out.  A field
added to, removed from or reordered in only one side fails here instead of
mis-marshalling an option at run time."""
import ctypes
import pathlib
import shutil
import subprocess

import pytest

ROOT = pathlib.Path(__file__).resolve().parents[1]


def _structs():
    from paper_1306_1392_b300 import _lib
    return [getattr(_lib, n) for n in ("pyhst_geometry", "pyhst_preproc", "pyhst_tv_opts", "pyhst_tv_item",
                                       "pyhst_patch_problem")]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no host C compiler")
def test_ctypes_structures_match_the_header(tmp_path):
    structs = _structs()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pyhst.h"', "int main(void) {"]
    for S in structs:
        n = S.__name__
        lines.append(f'    printf("{n} sizeof %zu\\n", sizeof({n}));')
        for f, _t in S._fields_:
            lines.append(f'    printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", str(ROOT / "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for S in structs:
        n = S.__name__
        assert got[(n, "sizeof")] == ctypes.sizeof(S), n
        for f, _t in S._fields_:
            assert got[(n, f)] == getattr(S, f).offset, (n, f)
