"""Python binding of librix (ctypes; argument marshalling only).

Every function forwards to the C entry point of the same name in
``include/rix.h``; device buffers are torch CUDA tensors passed by
``data_ptr()`` together with the current CUDA stream.  There is no CPU
fallback: if the shared library cannot be loaded, import fails.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librix.so")

RIX_OK, RIX_EINVAL, RIX_ENOMEM, RIX_ECUDA, RIX_ENOTSYM, RIX_ETIMEOUT, RIX_EUNSUPPORTED, RIX_ESTATE = range(8)
RIX_FP64, RIX_MIXED_BF16 = 0, 1
RIX_LIST_C, RIX_LIST_V, RIX_LIST_D, RIX_LIST_K = 0, 1, 2, 3
PRECISIONS = {"fp64": RIX_FP64, "mixed": RIX_MIXED_BF16, "bf16": RIX_MIXED_BF16}


class RixError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"rix status {status}: {msg}")


class _System(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("xyz_bohr", ctypes.c_void_p), ("species", ctypes.c_void_p),
                ("n_species", ctypes.c_int32), ("nbas_per_species", ctypes.c_void_p),
                ("naux_per_species", ctypes.c_void_p), ("cell_bohr", ctypes.c_void_p),
                ("cutoff_bohr", ctypes.c_double), ("screen_tau", ctypes.c_double),
                ("n_pairs", ctypes.c_int64), ("pairs", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("max_workspace_bytes", ctypes.c_int64), ("verbose", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("backward", ctypes.c_int32), ("block_atoms", ctypes.c_int32),
                ("n_slices_regrouped", ctypes.c_int32), ("reuse_forward", ctypes.c_int32),
                ("product_tau", ctypes.c_double), ("deterministic", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int64), ("n_pairs", ctypes.c_int64), ("n_pairs2", ctypes.c_int64),
                ("n_kblocks", ctypes.c_int64), ("c_elems", ctypes.c_int64), ("v_elems", ctypes.c_int64),
                ("d_elems", ctypes.c_int64), ("k_elems", ctypes.c_int64), ("flops_fp64", ctypes.c_double),
                ("flops_stage", ctypes.c_double * 6), ("min_bytes", ctypes.c_double),
                ("tensor_flops", ctypes.c_double), ("workspace_bytes", ctypes.c_int64),
                ("n_row_blocks", ctypes.c_int32), ("flops_term2", ctypes.c_double),
                ("tensor_flops_stage", ctypes.c_double * 5), ("launches_build", ctypes.c_int32),
                ("flops_term1_tc", ctypes.c_double), ("flops_z_tc", ctypes.c_double),
                ("tz_bytes", ctypes.c_int64), ("flops_t_tc", ctypes.c_double), ("nbasis", ctypes.c_int64)]


_lib = None


def load():
    """Load librix.so (built by ``paper_2403_10343_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librix.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.rix_setup.argtypes = [ctypes.POINTER(_System), ctypes.POINTER(_Options), ctypes.POINTER(P)]
    lib.rix_layout.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.POINTER(ctypes.c_int64)),
                               ctypes.POINTER(ctypes.POINTER(ctypes.c_int64))]
    lib.rix_layout_sizes.argtypes = [P] + [ctypes.POINTER(ctypes.c_int64)] * 4
    lib.rix_set_CV.argtypes = [P, P, P, P]
    lib.rix_build_K.argtypes = [P, P, P, P]
    lib.rix_energy.argtypes = [P, P, P, P, P]
    lib.rix_energy_noalloc.argtypes = [P, P, P, P, P]
    lib.rix_backward.argtypes = [P, P, ctypes.c_double, P, P, P, P]
    lib.rix_fold_gamma.argtypes = [P, P, P, P]
    lib.rix_stats.argtypes = [P, ctypes.POINTER(_Stats)]
    lib.rix_gemm_sliced.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]
    lib.rix_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)]
    lib.rix_autotune.argtypes = [P, P, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int32), P]
    lib.rix_count_flops.argtypes = [P, P, ctypes.POINTER(ctypes.c_double), P]
    lib.rix_check.argtypes = [P, P]
    lib.rix_build_K_delta.argtypes = [P, P, P, P]
    lib.rix_force_stress.argtypes = [P, ctypes.c_int32, P, P, P, P, P, P, P]
    lib.rix_fit_C.argtypes = [P, P, P, ctypes.c_double, P, P]
    lib.rix_gemm_profile.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                     ctypes.POINTER(ctypes.c_int64)]
    lib.rix_bloch.argtypes = [P, P, ctypes.c_int32, P, P, P]
    lib.rix_build_K_spin.argtypes = [P, ctypes.c_int32, P, P, P]
    lib.rix_energy_spin.argtypes = [P, ctypes.c_int32, P, P, P, P]
    lib.rix_test_stalled_gemm.argtypes = [P, ctypes.c_int64, P]
    lib.rix_strerror.restype = ctypes.c_char_p
    lib.rix_strerror.argtypes = [I]
    lib.rix_last_error.restype = ctypes.c_char_p
    lib.rix_last_error.argtypes = [P]
    lib.rix_destroy.argtypes = [P]
    for f in ("rix_setup", "rix_layout", "rix_layout_sizes", "rix_set_CV", "rix_build_K", "rix_energy",
              "rix_energy_noalloc",
              "rix_backward", "rix_fold_gamma", "rix_stats", "rix_stage_times", "rix_gemm_sliced",
              "rix_autotune", "rix_count_flops", "rix_check", "rix_test_stalled_gemm", "rix_bloch",
              "rix_build_K_spin", "rix_energy_spin", "rix_build_K_delta", "rix_force_stress",
              "rix_gemm_profile", "rix_fit_C"):
        getattr(lib, f).restype = I
    _lib = lib
    return lib


def _check(st, ctx=None):
    if st != RIX_OK:
        lib = load()
        msg = lib.rix_strerror(st).decode()
        if ctx is not None:
            msg += ": " + lib.rix_last_error(ctx).decode()
        raise RixError(st, msg)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, name, min_numel=1, device=None):
    """Device pointer of a contiguous float64 CUDA tensor holding at least min_numel elements.

    The kernels index these buffers by the context's layout, so a wrong dtype, a
    short tensor or one on another GPU would make them read or write out of bounds.
    """
    if t is None:
        return None
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64, got {t.dtype}")
    if t.numel() < min_numel:
        raise ValueError(f"{name} holds {t.numel()} elements, the layout needs {min_numel}")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    return ctypes.c_void_p(t.data_ptr())


def _sizes(ctx):
    """(c_elems, v_elems, d_elems, k_elems) of a context."""
    return layout_sizes(ctx)


def setup(xyz_bohr, species, nbas, naux, cell_bohr=None, cutoff_bohr=0.0, screen_tau=0.0,
          precision="fp64", n_slices=0, max_workspace_bytes=0, verbose=0, profile=0, backward=0,
          block_atoms=0, n_slices_regrouped=0, pairs=None, reuse_forward=0, product_tau=0.0,
          deterministic=0):
    """rix_setup: returns an opaque context handle (int).  pairs: optional [n, 5] (A, B, n1, n2, n3)."""
    lib = load()
    keep = [np.ascontiguousarray(xyz_bohr, dtype=np.float64), np.ascontiguousarray(species, dtype=np.int32),
            np.ascontiguousarray(nbas, dtype=np.int32), np.ascontiguousarray(naux, dtype=np.int32)]
    cell = None if cell_bohr is None else np.ascontiguousarray(cell_bohr, dtype=np.float64)
    pl = None if pairs is None else np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 5)
    sysd = _System(len(keep[1]), keep[0].ctypes.data, keep[1].ctypes.data, len(keep[2]), keep[2].ctypes.data,
                   keep[3].ctypes.data, None if cell is None else cell.ctypes.data,
                   float(cutoff_bohr), float(screen_tau), 0 if pl is None else len(pl),
                   None if pl is None else pl.ctypes.data)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    opt = _Options(prec, int(n_slices), int(max_workspace_bytes), int(verbose), int(profile), int(backward),
                   int(block_atoms), int(n_slices_regrouped), int(reuse_forward), float(product_tau),
                   int(deterministic))
    h = ctypes.c_void_p()
    _check(lib.rix_setup(ctypes.byref(sysd), ctypes.byref(opt), ctypes.byref(h)))
    return h.value


def layout(ctx, which):
    """rix_layout: (keys int64[n], offsets int64[n+1]) copied to numpy."""
    lib = load()
    n = ctypes.c_int64()
    k = ctypes.POINTER(ctypes.c_int64)()
    o = ctypes.POINTER(ctypes.c_int64)()
    _check(lib.rix_layout(ctx, which, ctypes.byref(n), ctypes.byref(k), ctypes.byref(o)), ctx)
    keys = np.ctypeslib.as_array(k, shape=(n.value,)).copy() if n.value else np.zeros(0, np.int64)
    offs = np.ctypeslib.as_array(o, shape=(n.value + 1,)).copy()
    return keys, offs


def layout_sizes(ctx):
    lib = load()
    v = [ctypes.c_int64() for _ in range(4)]
    _check(lib.rix_layout_sizes(ctx, *[ctypes.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def _any_ptr(x, name):
    """Device tensor, or a host array (numpy or CPU tensor) for rix_set_CV."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError(f"{name} must be a contiguous float64 array")
        return ctypes.c_void_p(x.ctypes.data)
    if not x.is_cuda:
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    return _dptr(x, name)


def _host_numel(x):
    return x.size if isinstance(x, np.ndarray) else x.numel()


def set_CV(ctx, C, V, stream=None):
    """rix_set_CV; C and V may be CUDA tensors or host arrays (copied either way)."""
    c, v, _, _ = _sizes(ctx)
    for x, name, n in ((C, "C", c), (V, "V", v)):
        if _host_numel(x) < n:
            raise ValueError(f"{name} holds {_host_numel(x)} elements, the layout needs {n}")
    _check(load().rix_set_CV(ctx, _any_ptr(C, "C"), _any_ptr(V, "V"), _stream(stream)), ctx)


def build_K(ctx, D, K, stream=None):
    _, _, d, k = _sizes(ctx)
    _check(load().rix_build_K(ctx, _dptr(D, "D", d), _dptr(K, "K", k, D.device), _stream(stream)), ctx)


def build_K_delta(ctx, dD, K, stream=None):
    """rix_build_K_delta: K += K(dD) (incremental build)."""
    _, _, d, k = _sizes(ctx)
    _check(load().rix_build_K_delta(ctx, _dptr(dD, "dD", d), _dptr(K, "K", k, dD.device), _stream(stream)), ctx)


def energy(ctx, D, K, Ex, stream=None):
    _, _, d, k = _sizes(ctx)
    _check(load().rix_energy(ctx, _dptr(D, "D", d), _dptr(K, "K", k, D.device), _dptr(Ex, "Ex", 1, D.device),
                             _stream(stream)), ctx)


def energy_noalloc(ctx, D, K, Ex, stream=None):
    """rix_energy_noalloc: the energy reduction without any device allocation."""
    _, _, d, k = _sizes(ctx)
    _check(load().rix_energy_noalloc(ctx, _dptr(D, "D", d), _dptr(K, "K", k, D.device),
                                     _dptr(Ex, "Ex", 1, D.device), _stream(stream)), ctx)


def backward(ctx, D, gEx, dD=None, dC=None, dV=None, stream=None):
    c, v, d, _ = _sizes(ctx)
    dev = D.device
    _check(load().rix_backward(ctx, _dptr(D, "D", d), float(gEx), _dptr(dD, "dD", d, dev), _dptr(dC, "dC", c, dev),
                               _dptr(dV, "dV", v, dev), _stream(stream)), ctx)


def bloch(ctx, K, kfrac, Kk, stream=None):
    """rix_bloch: Kk (complex128 CUDA tensor [n_k, nbasis, nbasis]) = Bloch sums of K at kfrac [n_k, 3]."""
    import torch
    kf = np.ascontiguousarray(kfrac, dtype=np.float64).reshape(-1, 3)
    nbasis = int(stats(ctx)["nbasis"])
    if Kk.dtype != torch.complex128 or not Kk.is_cuda or not Kk.is_contiguous():
        raise ValueError("Kk must be a contiguous complex128 CUDA tensor")
    if Kk.numel() < len(kf) * nbasis * nbasis:
        raise ValueError("Kk is too small for n_k nbasis x nbasis matrices")
    _, _, _, k = _sizes(ctx)
    _check(load().rix_bloch(ctx, _dptr(K, "K", k), len(kf), kf.ctypes.data, ctypes.c_void_p(Kk.data_ptr()),
                            _stream(stream)), ctx)


def build_K_spin(ctx, D, K, n_spin=2, stream=None):
    """rix_build_K_spin: D [n_spin * d_elems], K [n_spin * k_elems] (per-spin arrays back to back)."""
    _, _, d, k = _sizes(ctx)
    _check(load().rix_build_K_spin(ctx, int(n_spin), _dptr(D, "D", n_spin * d), _dptr(K, "K", n_spin * k, D.device),
                                   _stream(stream)), ctx)


def energy_spin(ctx, D, K, Ex, n_spin=2, stream=None):
    _, _, d, k = _sizes(ctx)
    _check(load().rix_energy_spin(ctx, int(n_spin), _dptr(D, "D", n_spin * d), _dptr(K, "K", n_spin * k, D.device),
                                  _dptr(Ex, "Ex", 1, D.device), _stream(stream)), ctx)


def force_stress(ctx, c, dEdC, dEdV, dCdr_c, dVdr_c, F=None, stress=None, stream=None):
    """rix_force_stress: component c of the forces [n_atoms] and row c of the stress [3] (device tensors)."""
    cel, vel, _, _ = _sizes(ctx)
    nat = int(stats(ctx)["n_atoms"])
    dev = (dEdC if dEdC is not None else dEdV).device
    _check(load().rix_force_stress(ctx, int(c), _dptr(dEdC, "dEdC", cel), _dptr(dEdV, "dEdV", vel, dev),
                                   _dptr(dCdr_c, "dCdr_c", cel, dev), _dptr(dVdr_c, "dVdr_c", vel, dev),
                                   _dptr(F, "F", nat, dev), _dptr(stress, "stress", 3, dev), _stream(stream)), ctx)


def fit_C(ctx, V, eri, lam=0.0, C=None, stream=None):
    """rix_fit_C: RI coefficients from the three-centre integrals (packed C layout) and the metric V."""
    import torch
    cel, vel, _, _ = _sizes(ctx)
    if C is None:
        C = torch.empty(cel, dtype=torch.float64, device=eri.device)
    _check(load().rix_fit_C(ctx, _dptr(V, "V", vel), _dptr(eri, "eri", cel, V.device), float(lam),
                            _dptr(C, "C", cel, V.device), _stream(stream)), ctx)
    return C


def check(ctx, stream=None):
    """rix_check: synchronise and raise if a bounded device wait of the context gave up."""
    _check(load().rix_check(ctx, _stream(stream)), ctx)


def stalled_gemm(wait_ns, ctx=None, stream=None):
    """rix_test_stalled_gemm: the status (ctx None: RIX_ETIMEOUT when the timeout path worked)."""
    return load().rix_test_stalled_gemm(ctx, int(wait_ns), _stream(stream))


def autotune(ctx, D, cache_path=None, stream=None):
    """rix_autotune: returns the chosen tile budgets (doubles) of k_X12, k_Z, k_X34."""
    out = (ctypes.c_int32 * 3)()
    path = None if cache_path is None else os.fsencode(cache_path)
    _, _, d, _ = _sizes(ctx)
    _check(load().rix_autotune(ctx, _dptr(D, "D", d), path, out, _stream(stream)), ctx)
    return tuple(out)


COUNT_KEYS = ("T", "U2", "X12", "Z", "X34", "sym", "term2", "term1_tc", "z_tc", "t_tc")


def count_flops(ctx, D, stream=None):
    """rix_count_flops: FLOPs of one build with this D after block screening, by stage."""
    out = (ctypes.c_double * 10)()
    _, _, d, _ = _sizes(ctx)
    _check(load().rix_count_flops(ctx, _dptr(D, "D", d), out, _stream(stream)), ctx)
    return dict(zip(COUNT_KEYS, out))


def fold_gamma(ctx, K, Kdense, stream=None):
    _, _, _, k = _sizes(ctx)
    nbasis = int(stats(ctx)["nbasis"])
    _check(load().rix_fold_gamma(ctx, _dptr(K, "K", k), _dptr(Kdense, "Kdense", nbasis * nbasis, K.device),
                                 _stream(stream)), ctx)


def stats(ctx):
    s = _Stats()
    _check(load().rix_stats(ctx, ctypes.byref(s)), ctx)
    d = {f: getattr(s, f) for f, _ in _Stats._fields_ if f not in ("flops_stage", "tensor_flops_stage")}
    d["flops_stage"] = list(s.flops_stage)
    d["tensor_flops_stage"] = list(s.tensor_flops_stage)
    return d


def gemm_sliced(A, B, n_slices, C=None, stream=None):
    """rix_gemm_sliced: C = A @ B (FP64 CUDA matrices) on the BF16 tensor cores."""
    import torch
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    if tuple(C.shape) != (M, N):
        raise ValueError("C must be M x N")
    _check(load().rix_gemm_sliced(_dptr(A, "A", M * K), A.stride(0), _dptr(B, "B", K * N, A.device), B.stride(0),
                                  _dptr(C, "C", M * N, A.device), C.stride(0), M, N, K, int(n_slices),
                                  _stream(stream)))
    return C


STAGES = ("flags", "T", "U2", "X12", "TC12", "Z", "X34", "sym")


def stage_times(ctx):
    """rix_stage_times: (dict stage -> summed ms, number of builds)."""
    ms = (ctypes.c_double * len(STAGES))()
    nb = ctypes.c_int32()
    _check(load().rix_stage_times(ctx, ms, len(STAGES), ctypes.byref(nb)), ctx)
    return dict(zip(STAGES, list(ms))), nb.value


def gemm_profile(ctx):
    """rix_gemm_profile: (summed ms, launches, K stages) of the sliced-GEMM launches since the last call."""
    ms, n, ch = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().rix_gemm_profile(ctx, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(ch)), ctx)
    return ms.value, n.value, ch.value


def destroy(ctx):
    if ctx:
        load().rix_destroy(ctx)


class Exchange:
    """Convenience owner of one rix context plus its device-resident C and V."""

    def __init__(self, xyz_bohr, species, nbas, naux, cell_bohr=None, cutoff_bohr=0.0, screen_tau=0.0,
                 precision="fp64", n_slices=0, max_workspace_bytes=0, verbose=0, profile=0, backward=0,
                 block_atoms=0, n_slices_regrouped=0, pairs=None, reuse_forward=0, product_tau=0.0,
                 deterministic=0):
        self.ctx = setup(xyz_bohr, species, nbas, naux, cell_bohr, cutoff_bohr, screen_tau, precision,
                         n_slices, max_workspace_bytes, verbose, profile, backward, block_atoms,
                         n_slices_regrouped, pairs, reuse_forward, product_tau, deterministic)
        self.c_elems, self.v_elems, self.d_elems, self.k_elems = layout_sizes(self.ctx)

    @classmethod
    def from_system(cls, system, **kw):
        return cls(system.xyz, system.species, system.nbas, system.naux, system.cell, system.cutoff,
                   system.tau, **kw)

    def pair_keys(self):
        return layout(self.ctx, RIX_LIST_C)[0]

    def k_keys(self):
        return layout(self.ctx, RIX_LIST_K)[0]

    def set_CV(self, C, V, stream=None):
        self._cv_stamp = None  # the autograd wrapper reloads on its next call
        set_CV(self.ctx, C, V, stream)

    def check(self, stream=None):
        check(self.ctx, stream)

    def autotune(self, D, cache_path=None, stream=None):
        return autotune(self.ctx, D, cache_path, stream)

    def count_flops(self, D, stream=None):
        return count_flops(self.ctx, D, stream)

    def build_K(self, D, K=None, stream=None):
        import torch
        if K is None:
            K = torch.empty(self.k_elems, dtype=torch.float64, device=D.device)
        build_K(self.ctx, D, K, stream)
        return K

    def energy(self, D, K, Ex=None, stream=None):
        import torch
        if Ex is None:
            Ex = torch.empty(1, dtype=torch.float64, device=D.device)
        energy(self.ctx, D, K, Ex, stream)
        return Ex

    def backward(self, D, gEx, dD=None, dC=None, dV=None, want=("D", "C", "V"), stream=None):
        """Gradients of gEx * E_x; allocates the requested outputs when not given."""
        import torch
        dev = D.device
        if dD is None and "D" in want:
            dD = torch.empty(self.d_elems, dtype=torch.float64, device=dev)
        if dC is None and "C" in want:
            dC = torch.empty(self.c_elems, dtype=torch.float64, device=dev)
        if dV is None and "V" in want:
            dV = torch.empty(self.v_elems, dtype=torch.float64, device=dev)
        backward(self.ctx, D, gEx, dD, dC, dV, stream)
        return dD, dC, dV

    def fold_gamma(self, K, nbasis, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((nbasis, nbasis), dtype=torch.float64, device=K.device)
        fold_gamma(self.ctx, K, out, stream)
        return out

    def stats(self):
        return stats(self.ctx)

    def stage_times(self):
        return stage_times(self.ctx)

    def gemm_profile(self):
        return gemm_profile(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
