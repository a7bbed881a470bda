"""The ctypes structures of the Python binding (paper_1306_2150_gb300/lr.py)
against the C structs of include/lrpoisson.h: a small C program compiled
against the header reports every struct's size and every field's offset,
which must equal ctypes' (CPU only; gcc)."""
import json
import os
import shutil
import subprocess
import tempfile

import pytest

from paper_1306_2150_gb300 import lr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"lr_mat": lr.LrMat, "lr_tucker": lr.LrTucker, "lr_options": lr.LrOptions,
           "lr_tune": lr.LrTune, "lr_info": lr.LrInfo}


@pytest.fixture(scope="module")
def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lrpoisson.h"', "int main(void) {",
             '  printf("{");']
    first = True
    for cname, cls in STRUCTS.items():
        for fname, _ in cls._fields_:
            sep = "" if first else ","
            lines.append(f'  printf("{sep}\\"{cname}.{fname}\\": %zu", offsetof({cname}, {fname}));')
            first = False
        lines.append(f'  printf(",\\"{cname}\\": %zu", sizeof({cname}));')
    lines += ['  printf("}\\n");', "  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return json.loads(out)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_struct_matches_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert c_layout[cname] == __import__("ctypes").sizeof(cls), cname
    for fname, _ in cls._fields_:
        assert c_layout[f"{cname}.{fname}"] == getattr(cls, fname).offset, (cname, fname)
