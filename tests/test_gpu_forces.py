"""Force and stress chain on the GPU (rix_backward + rix_force_stress) against the oracle.

* A water dimer (cluster): forces from the device adjoint and rix_force_stress
  equal the oracle chain (oracle/forces.py) fed with the dense-definition
  adjoint (oracle/grad.py) and the same dC/dr, dV/dr, to 1e-10 of the largest
  force.
* A periodic cell with atoms near the faces: forces and the stress row of
  every Cartesian component equal central differences of the oracle energy
  with C and V regenerated at the displaced / strained geometry (same random
  draws), to 1e-6 of the largest value (the difference's own error).
Both the FP64 and the mixed path (mixed forward recompute, FP64 adjoint).
"""
import dataclasses

import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.forces import forces_stress
from oracle.oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402
from test_oracle_forces import _adjoint_dense, _energy  # noqa: E402
from test_oracle_images import _base  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _gpu_forces(s, pk, prec):
    ex = rix.Exchange.from_system(s, precision=prec, backward=1)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    D = _dev(pk.D)
    _, dEdC, dEdV = ex.backward(D, 1.0, want=("C", "V"))
    dC, dV = pk.gen_derivatives()
    F = torch.empty((3, s.n_atoms), dtype=torch.float64, device="cuda")
    st = torch.empty((3, 3), dtype=torch.float64, device="cuda") if s.cell is not None else None
    for c in range(3):
        rix.force_stress(ex.ctx, c, dEdC, dEdV, _dev(dC[c]), _dev(dV[c]), F[c],
                         None if st is None else st[c])
    torch.cuda.synchronize()
    out = F.cpu().numpy().T, (None if st is None else st.cpu().numpy())
    ex.close()
    return out


def _dimer():
    xyz, spc = S._waters(np.array([[0.0, 0.0, 0.0], [2.9, 0.4, -0.3]]), 7)
    nb, na = S._species_arrays(["O", "H"])
    return S.System(name="dimer", seed=7, xyz=ri.ang2bohr(xyz), species=spc, species_names=["O", "H"], nbas=nb,
                    naux=na, sigma=S._aux_widths(7, ["O", "H"]), cell=None, cutoff=0.0, tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cluster_forces_against_oracle_chain(prec):
    s = _dimer()
    pk = ri.generate(s)
    dEdC, dEdV = _adjoint_dense(s, pk)
    dC, dV = pk.gen_derivatives()
    F_ref, _ = forces_stress(s, pk, dEdC, dEdV, dC, dV)
    F, _ = _gpu_forces(s, pk, prec)
    err = np.abs(F - F_ref).max() / np.abs(F_ref).max()
    print(f"{prec}: dimer forces vs oracle chain {err:.2e}")
    assert err < (1e-10 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_periodic_forces_and_stress_against_finite_differences(prec):
    s, pk = _base()
    F, st = _gpu_forces(s, pk, prec)
    h = 1e-4
    Fs = np.abs(F).max()
    for atom, c in ((0, 0), (2, 1), (4, 2)):
        e = []
        for sg in (1, -1):
            x = s.xyz.copy()
            x[atom, c] += sg * h
            s2 = dataclasses.replace(s, xyz=x)
            assert np.array_equal(ri.pair_list(s2)[0], pk.keys)
            e.append(_energy(s2, pk.D))
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - F[atom, c]) < 1e-6 * Fs, (atom, c, fd, F[atom, c])
    omega = abs(np.linalg.det(s.cell))
    ss = np.abs(st).max()
    for a, b in ((0, 0), (1, 2), (2, 1)):
        e = []
        for sg in (1, -1):
            eps = np.zeros((3, 3))
            eps[a, b] = sg * h
            M = np.eye(3) + eps                       # r -> (1 + eps) r
            s2 = dataclasses.replace(s, xyz=s.xyz @ M.T, cell=s.cell @ M.T)
            assert np.array_equal(ri.pair_list(s2)[0], pk.keys)
            e.append(_energy(s2, pk.D))
        fd = (e[0] - e[1]) / (2 * h) / omega
        print(f"{prec}: stress[{a}][{b}] chain {st[a, b]:.10e}, finite difference {fd:.10e}")
        assert abs(fd - st[a, b]) < 1e-6 * ss
