"""Bloch sums (Eq. 3) and collinear spin channels on the GPU against the oracle.

rix_bloch applied to the device K must equal the oracle's Bloch sum of the
oracle's K (written out from Eq. 3) at several k points, to the FP64 bar
(1e-12 relative to the largest element) for the FP64 path and the mixed bar
(1e-8) for the mixed path.  rix_build_K_spin / rix_energy_spin of a
spin-polarised density must equal the oracle's per-channel builds and
E_x = -1/2 sum_sigma Tr(D^sigma K^sigma).
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.kspace import bloch_sum, exchange_spin
from oracle.oracle import exchange

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402
from test_oracle_images import _base  # noqa: E402

KFRAC = np.array([[0, 0, 0], [0.5, 0, 0], [0.25, -0.125, 0.375], [0.5, 0.5, 0.5]])
TOL = {"fp64": (1e-12, 1e-12), "mixed": (1e-8, 1e-6)}


def _system(case):
    if case == "waters":
        return _base()
    s = S.perovskite(1, 1, 1, 31)
    s.cutoff = ri.ang2bohr(6.5)
    return s, ri.generate(s)


@pytest.mark.parametrize("case", ["waters", "perovskite"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_bloch_sums(case, prec):
    s, pk = _system(case)
    kk, K_ref, _, _ = exchange(s, pk)
    ref = bloch_sum(s, kk, K_ref, KFRAC)
    ex = rix.Exchange.from_system(s, precision=prec)
    dev = torch.device("cuda")
    C, V, D = (torch.from_numpy(x).to(dev) for x in (pk.C, pk.V, pk.D))
    ex.set_CV(C, V)
    K = ex.build_K(D)
    nbasis = s.nbasis
    Kk = torch.full((len(KFRAC), nbasis, nbasis), complex("nan"), dtype=torch.complex128, device=dev)
    rix.bloch(ex.ctx, K, KFRAC, Kk)
    # the Gamma point equals rix_fold_gamma
    Kg = ex.fold_gamma(K, nbasis)
    torch.cuda.synchronize()
    got = Kk.cpu().numpy()
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    print(f"{case} {prec}: Bloch sums max error {err:.2e} of the largest element")
    assert err < TOL[prec][0]
    # (the fold and the Bloch kernel sum a pair's images in different orders)
    assert np.abs(got[0].real - Kg.cpu().numpy()).max() < 1e-15 * scale and not got[0].imag.any()
    ex.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spin_channels(prec):
    s = ri.config(0)
    pk = ri.generate(s)
    Du, Dd = pk.gen_D_spin()
    kk, (Ku_ref, Kd_ref), E_ref = exchange_spin(s, pk, Du, Dd)
    ex = rix.Exchange.from_system(s, precision=prec)
    dev = torch.device("cuda")
    ex.set_CV(torch.from_numpy(pk.C).to(dev), torch.from_numpy(pk.V).to(dev))
    D2 = torch.from_numpy(np.concatenate([Du, Dd])).to(dev)
    K2 = torch.empty(2 * ex.k_elems, dtype=torch.float64, device=dev)
    Ex = torch.empty(1, dtype=torch.float64, device=dev)
    rix.build_K_spin(ex.ctx, D2, K2)
    rix.energy_spin(ex.ctx, D2, K2, Ex)
    torch.cuda.synchronize()
    K2 = K2.cpu().numpy()
    ktol, etol = TOL[prec]
    for got, ref in ((K2[:ex.k_elems], Ku_ref), (K2[ex.k_elems:], Kd_ref)):
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < ktol
    E = Ex.item()
    print(f"{prec}: spin-polarised E_x {E:.10f} Ha, oracle {E_ref:.10f}")
    assert abs(E - E_ref) < (etol * abs(E_ref) if prec == "fp64" else etol)
    ex.close()
