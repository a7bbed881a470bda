"""The C-ABI library builds, loads, and exports every symbol its header
declares; host-only behaviour without a GPU.  CPU only: no compute calls."""
import ctypes
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADER = ROOT / "include" / "lrpoisson.h"


def _declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(lr_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1306_2150_gb300 import build, lr
    build.build()
    return lr.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("lr_poisson2d", "lr_truncate", "lr_dst1", "lr_create", "lr_destroy", "lr_get_info"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1306_2150_gb300 import lr
    names = _declared_functions()
    assert sorted(lr.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", lr.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (lr_[a-z0-9_]+)$", out, flags=re.M))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_library_targets_sm103a():
    from paper_1306_2150_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_options_defaults_and_status_strings(lib):
    from paper_1306_2150_gb300 import lr
    o = lr.lr_options_default()
    assert o.prec == lr.LR_MIXED and o.op == lr.LR_OP_5PT
    assert o.eps == 1e-6 and o.rmax == 64 and o.aca_tol_factor == 1.0 and o.probes == 16
    assert lr.status_string(lr.LR_ENOCONV) == "LR_ENOCONV"
    assert ctypes.sizeof(lr.LrMat) == 4 * 5 + 4 + 3 * 8  # 5 ints + pad + 3 pointers


def test_null_arguments_rejected_without_device(lib):
    from paper_1306_2150_gb300 import lr
    assert lib.lr_create(None, None) == lr.LR_EINVAL
    assert lib.lr_destroy(None) == lr.LR_EINVAL
    assert lib.lr_poisson2d(None, None, None, None) == lr.LR_EINVAL
    assert lib.lr_last_error(None) == b"null handle"
    rows = (ctypes.c_int * 2)(0, 1)
    assert lib.lr_maxvol(None, None, 4, 2, 4, 0.01, 8, rows, None, None) == lr.LR_EINVAL
