"""ctypes wrapper of the plain-C FP64 oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke`` and the benchmark's CPU-baseline leg
may import this module.  The library under test never does.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rix_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (-O2, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P,
                                       ctypes.c_double, ctypes.c_double]
            lib.orc_npairs.restype = ctypes.c_int64
            lib.orc_npairs.argtypes = [P]
            lib.orc_pairs.argtypes = [P, P]
            lib.orc_size.restype = ctypes.c_int64
            lib.orc_size.argtypes = [P, ctypes.c_int]
            lib.orc_set_data.argtypes = [P, P, P, P]
            lib.orc_kpattern.restype = ctypes.c_int64
            lib.orc_kpattern.argtypes = [P, ctypes.c_int, P]
            lib.orc_kkeys.argtypes = [P, P]
            lib.orc_ksize.restype = ctypes.c_int64
            lib.orc_ksize.argtypes = [P]
            lib.orc_build_K.restype = ctypes.c_int
            lib.orc_build_K.argtypes = [P, P]
            lib.orc_energy.restype = ctypes.c_double
            lib.orc_energy.argtypes = [P, P, P]
            lib.orc_destroy.argtypes = [P]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_terms.argtypes = [P, ctypes.c_int]
            lib.orc_build_K_ex.restype = ctypes.c_int
            lib.orc_build_K_ex.argtypes = [P, P, ctypes.c_int]
            lib.orc_kpattern_blocks.restype = ctypes.c_int64
            lib.orc_kpattern_blocks.argtypes = [P, ctypes.c_int64, P]
            lib.orc_flops.restype = ctypes.c_double
            lib.orc_flops.argtypes = [P]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Oracle:
    """Oracle bound to one system; builds its own pair list."""

    def __init__(self, system):
        lib = _load()
        self.lib = lib
        self.system = system
        self._xyz = np.ascontiguousarray(system.xyz, dtype=np.float64)
        self._sp = np.ascontiguousarray(system.species, dtype=np.int32)
        self._nb = np.ascontiguousarray(system.nbas, dtype=np.int32)
        self._na = np.ascontiguousarray(system.naux, dtype=np.int32)
        self._cell = None if system.cell is None else np.ascontiguousarray(system.cell, dtype=np.float64)
        h = lib.orc_create(len(self._sp), _ptr(self._xyz), _ptr(self._sp), len(self._nb),
                           _ptr(self._nb), _ptr(self._na), _ptr(self._cell),
                           float(system.cutoff), float(system.tau))
        if not h:
            raise RuntimeError("oracle: invalid system")
        self.h = h
        self._data = None

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    @staticmethod
    def threads():
        return _load().orc_threads()

    @staticmethod
    def set_threads(n):
        """Threads of the row loops (0: every processor)."""
        _load().orc_set_threads(int(n))

    def set_terms(self, mask):
        """Restrict the sum to a subset of the four terms (bit t-1 = term t)."""
        self.lib.orc_set_terms(self.h, int(mask))

    def pair_keys(self):
        n = self.lib.orc_npairs(self.h)
        k = np.empty(n, dtype=np.int64)
        self.lib.orc_pairs(self.h, _ptr(k))
        return k

    def sizes(self):
        return tuple(int(self.lib.orc_size(self.h, w)) for w in range(3))

    def set_data(self, C, V, D):
        C = np.ascontiguousarray(C, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        D = np.ascontiguousarray(D, dtype=np.float64)
        if (C.size, V.size, D.size) != self.sizes():
            raise ValueError("packed sizes do not match the oracle's pair list")
        self._data = (C, V, D)  # keep alive
        self.lib.orc_set_data(self.h, _ptr(C), _ptr(V), _ptr(D))

    def kpattern(self, rows=None):
        if rows is None:
            nk = self.lib.orc_kpattern(self.h, -1, None)
            self._rows = None
        else:
            r = np.ascontiguousarray(rows, dtype=np.int32)
            self._rows = r
            nk = self.lib.orc_kpattern(self.h, len(r), _ptr(r))
        k = np.empty(nk, dtype=np.int64)
        self.lib.orc_kkeys(self.h, _ptr(k))
        return k

    def kpattern_blocks(self, keys):
        """Sampled mode: only the listed K blocks (A, E', n); returns them sorted."""
        k = np.ascontiguousarray(keys, dtype=np.int64)
        self._rows = None
        self._sampled = k
        n = self.lib.orc_kpattern_blocks(self.h, len(k), k.ctypes.data_as(ctypes.c_void_p))
        out = np.empty(n, dtype=np.int64)
        self.lib.orc_kkeys(self.h, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def build_K(self, dry=False):
        """K for the rows of the last kpattern(); dry=True only counts the work."""
        K = np.empty(self.lib.orc_ksize(self.h), dtype=np.float64)
        if self.lib.orc_build_K_ex(self.h, _ptr(K), 1 if dry else 0) != 0:
            raise RuntimeError("oracle: build_K before set_data/kpattern")
        return K

    def flops(self):
        """FLOPs (2 per multiply-add) the last build_K did or, dry, would do."""
        return self.lib.orc_flops(self.h)

    def energy(self, K, per_row=False):
        nr = self.system.n_atoms if self._rows is None else len(self._rows)
        pr = np.empty(nr, dtype=np.float64)
        e = self.lib.orc_energy(self.h, _ptr(np.ascontiguousarray(K)), _ptr(pr))
        return (e, pr) if per_row else e


def exchange(system, packed, rows=None):
    """Convenience: (K keys, K packed, E_x) from the oracle on the packed inputs."""
    o = Oracle(system)
    if not np.array_equal(o.pair_keys(), packed.keys):
        raise AssertionError("oracle pair list differs from the generator's")
    o.set_data(packed.C, packed.V, packed.D)
    kk = o.kpattern(rows)
    K = o.build_K()
    return kk, K, o.energy(K), o
