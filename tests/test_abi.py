"""The C-ABI library loads and exports every entry point include/rix.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rix.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rix_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("rix_setup", "rix_layout", "rix_set_CV", "rix_build_K", "rix_energy", "rix_backward",
              "rix_fold_gamma", "rix_stats", "rix_strerror", "rix_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2403_10343_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    from paper_2403_10343_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.rix_strerror.restype = ctypes.c_char_p
    assert lib.rix_strerror(0) == b"ok"
    assert lib.rix_strerror(4).startswith(b"C or V")
