"""Incremental (Delta D) builds and the full-range (PBE0) Coulomb metric on the GPU.

* rix_build_K_delta: K(D1) followed by K += K(D2 - D1) equals the oracle's
  K(D2) (no screening), FP64 and mixed; with block screening the density
  change confined to one molecule (every other block of dD below tau) gives
  the oracle's K(D1) + K(dD) with the same screening, and the stages that
  read D (T and Z) skip the screened blocks (rix_count_flops of dD is a
  fraction of that of D there).
* PBE0: V from the full-range metric erf(R/g1)/R (no decay with distance
  beyond the cutoff) through the same build, against the oracle at the FP64
  and mixed bars.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.oracle import Oracle, exchange

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402

TOL = {"fp64": (1e-12, 1e-12), "mixed": (1e-8, 1e-6)}


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _oracle_K(s, pk, D):
    o = Oracle(s)
    o.set_data(pk.C, pk.V, D)
    kk = o.kpattern()
    K = o.build_K()
    return kk, K, o.energy(K)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_delta_build_equals_full_build(prec):
    s = ri.config(0)
    pk = ri.generate(s)
    _, Dd = pk.gen_D_spin()
    D2 = pk.D
    D1 = 0.9 * D2 + 0.2 * Dd                           # not proportional to D2
    kk, K_ref, E_ref = _oracle_K(s, pk, D2)
    ex = rix.Exchange.from_system(s, precision=prec)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    K = ex.build_K(_dev(D1))
    rix.build_K_delta(ex.ctx, _dev(D2 - D1), K)
    E = ex.energy(_dev(D2), K)
    torch.cuda.synchronize()
    err = _rel(K.cpu().numpy(), K_ref)
    print(f"{prec}: K(D1) + K(D2 - D1) vs oracle K(D2): {err:.2e}, dE {E.item() - E_ref:.2e} Ha")
    assert err < TOL[prec][0]
    ex.close()


def test_delta_build_with_screening_skips_blocks():
    s = ri.config(1)                                   # 8 A cutoff, tau = 1e-10
    pk = ri.generate(s)
    _, Dd = pk.gen_D_spin()
    # density change on the pairs touching the first water; elsewhere below tau
    near = np.isin(pk.A, [0, 1, 2]) | np.isin(pk.B, [0, 1, 2])
    dD = np.zeros_like(pk.D)
    tiny = np.zeros_like(pk.D)
    for p in range(pk.n_pairs):
        sl = slice(pk.offD[p], pk.offD[p + 1])
        if near[p]:
            dD[sl] = 1e-2 * (Dd[sl] - 0.5 * pk.D[sl])     # one orbital of every five emptied
        else:
            tiny[sl] = 1e-12 * np.sign(pk.D[sl])       # |x| < tau: screened out by both sides
    dD = dD + tiny
    rows = [0, 1, 2, 90, 91, 92]
    ex = rix.Exchange.from_system(s)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    D1 = _dev(pk.D)
    K = ex.build_K(D1)
    K1 = K.clone()
    rix.build_K_delta(ex.ctx, _dev(dD), K)
    # the stages that read D directly (T and Z) skip the screened blocks of dD
    f_full = sum(ex.count_flops(D1)[k] for k in ("T", "Z"))
    f_delta = sum(ex.count_flops(_dev(dD))[k] for k in ("T", "Z"))
    torch.cuda.synchronize()
    got = (K - K1).cpu().numpy()
    o = Oracle(s)
    o.set_data(pk.C, pk.V, dD)
    kr = o.kpattern(rows)
    Kr = o.build_K()
    keys = ex.k_keys()
    A = ri.unpack_key(keys)[0]
    nb = s.nbas[s.species].astype(np.int64)
    E3 = ri.unpack_key(keys)[1]
    off = np.concatenate([[0], np.cumsum(nb[A] * nb[E3])])
    sel = np.nonzero(np.isin(A, rows))[0]
    sub = np.concatenate([got[off[x]:off[x + 1]] for x in sel])
    assert np.array_equal(keys[sel], kr)
    assert np.linalg.norm(Kr) > 0
    err = _rel(sub, Kr)
    print(f"delta build with screening: rows vs oracle K(dD) {err:.2e}; FLOPs {f_delta:.3e} of {f_full:.3e}")
    # K - K1 subtracts two numbers of K's size: its error is relative to K, not to K(dD)
    kscale = np.linalg.norm(np.concatenate([K1.cpu().numpy()[off[x]:off[x + 1]] for x in sel]))
    assert np.linalg.norm(sub - Kr) < 1e-12 * kscale
    assert f_delta < 0.5 * f_full
    ex.close()


def _pbc_selfimage():
    o = np.array([[1.0, 1.2, 0.8]])
    xyz, spc = S._waters(o, 11)
    nb, na = S._species_arrays(["O", "H"])
    return S.System(name="p", seed=11, xyz=ri.ang2bohr(xyz), species=spc, species_names=["O", "H"], nbas=nb,
                    naux=na, sigma=S._aux_widths(11, ["O", "H"]), cell=ri.ang2bohr(np.eye(3) * 4.6),
                    cutoff=ri.ang2bohr(4.8), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


@pytest.mark.parametrize("case", ["cluster24", "pbc_selfimage"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_range_kernel(case, prec):
    base = ri.config(0) if case == "cluster24" else _pbc_selfimage()
    s = ri.full_range(base)
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    ex = rix.Exchange.from_system(s, precision=prec)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    D = _dev(pk.D)
    K = ex.build_K(D)
    E = ex.energy(D, K).item()
    assert np.array_equal(ex.k_keys(), kk)
    err = _rel(K.cpu().numpy(), K_ref)
    print(f"PBE0 {case} {prec}: K {err:.2e}, E_x {E:.8f} (oracle {E_ref:.8f})")
    ktol, etol = TOL[prec]
    assert err < ktol
    assert abs(E - E_ref) < (etol * abs(E_ref) if prec == "fp64" else etol)
    ex.close()
