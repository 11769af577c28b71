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


def test_invalid_arguments_fail_before_any_device_work():
    """The documented argument checks return RIX_EINVAL without touching a GPU."""
    from paper_2403_10343_gb300 import build, rix
    lib = ctypes.CDLL(build.build())
    P = ctypes.c_void_p
    lib.rix_setup.argtypes = [ctypes.POINTER(rix._System), ctypes.POINTER(rix._Options), ctypes.POINTER(P)]
    out = P(123)
    assert lib.rix_setup(None, None, ctypes.byref(out)) == 1 and not out.value
    xyz = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    sp = (ctypes.c_int32 * 1)(0)
    nb, na = (ctypes.c_int32 * 1)(14), (ctypes.c_int32 * 1)(56)
    good = dict(n_atoms=1, xyz_bohr=ctypes.cast(xyz, P), species=ctypes.cast(sp, P), n_species=1,
                nbas_per_species=ctypes.cast(nb, P), naux_per_species=ctypes.cast(na, P), cell_bohr=None,
                cutoff_bohr=0.0, screen_tau=0.0)
    cell = (ctypes.c_double * 9)(10, 0, 0, 0, 10, 0, 0, 0, 10)
    bad_cases = [
        dict(good, n_atoms=0),                              # no atoms
        dict(good, species=ctypes.cast((ctypes.c_int32 * 1)(1), P)),  # species id out of range
        dict(good, cell_bohr=ctypes.cast(cell, P)),         # periodic cell without a cutoff
        dict(good, nbas_per_species=ctypes.cast((ctypes.c_int32 * 1)(65), P)),  # block above 64
        dict(good, xyz_bohr=ctypes.cast((ctypes.c_double * 3)(0.0, float("nan"), 0.0), P)),
    ]
    for kw in bad_cases:
        sysd = rix._System(**kw)
        assert lib.rix_setup(ctypes.byref(sysd), None, ctypes.byref(out)) == 1, kw
        assert not out.value
    opt = rix._Options(7, 0, 0, 0, 0, 0, 0)                # unknown precision
    sysd = rix._System(**good)
    assert lib.rix_setup(ctypes.byref(sysd), ctypes.byref(opt), ctypes.byref(out)) == 1
    lib.rix_stats.argtypes = [P, P]
    assert lib.rix_stats(None, None) == 1
    lib.rix_last_error.restype = ctypes.c_char_p
    lib.rix_last_error.argtypes = [P]
    assert lib.rix_last_error(None) == b""
    lib.rix_destroy.argtypes = [P]
    lib.rix_destroy(None)                                   # a no-op


def test_caller_pair_list_is_validated_before_any_device_work():
    """rix_system.pairs: out-of-range atoms, images in a cluster, duplicates and lists that are
    not symmetric are rejected with RIX_EINVAL (no GPU needed to get there)."""
    from paper_2403_10343_gb300 import build, rix
    lib = ctypes.CDLL(build.build())
    P = ctypes.c_void_p
    lib.rix_setup.argtypes = [ctypes.POINTER(rix._System), ctypes.POINTER(rix._Options), ctypes.POINTER(P)]
    xyz = (ctypes.c_double * 6)(0.0, 0.0, 0.0, 1.5, 0.0, 0.0)
    sp = (ctypes.c_int32 * 2)(0, 0)
    nb, na = (ctypes.c_int32 * 1)(5), (ctypes.c_int32 * 1)(16)
    out = P(123)

    def setup(rows, cell=None, n=None):
        arr = (ctypes.c_int32 * (5 * max(1, len(rows))))(*[v for r in rows for v in r])
        sysd = rix._System(2, ctypes.cast(xyz, P), ctypes.cast(sp, P), 1, ctypes.cast(nb, P), ctypes.cast(na, P),
                           cell, 10.0 if cell else 0.0, 0.0, len(rows) if n is None else n, ctypes.cast(arr, P))
        return lib.rix_setup(ctypes.byref(sysd), None, ctypes.byref(out))

    onsite = [(0, 0, 0, 0, 0), (1, 1, 0, 0, 0)]
    assert setup(onsite + [(0, 2, 0, 0, 0), (2, 0, 0, 0, 0)]) == 1          # atom out of range
    assert setup(onsite + [(0, 1, 1, 0, 0), (1, 0, -1, 0, 0)]) == 1         # image in a cluster
    assert setup(onsite + [(0, 1, 0, 0, 0), (0, 1, 0, 0, 0), (1, 0, 0, 0, 0)]) == 1  # duplicate
    assert setup(onsite + [(0, 1, 0, 0, 0)]) == 1                           # (1, 0) missing: not symmetric
    assert setup(onsite, n=0) == 1                                          # pointer without a count
    cell = (ctypes.c_double * 9)(30, 0, 0, 0, 30, 0, 0, 0, 30)
    assert setup(onsite + [(0, 1, 43, 0, 0), (1, 0, -43, 0, 0)], cell=ctypes.cast(cell, P)) == 1  # beyond +-42
    assert not out.value
