"""Pins of the force and stress chain (oracle/forces.py) against finite differences of the oracle energy.

The chain contracts the adjoint dE/dC, dE/dV (oracle/grad.py, from the dense
four-index definition of a cluster) with the generator's analytic dC/dr and
dV/dr (rix_inputs: C = g exp(-0.8 r), V = v(r; sigma)).  Independently, the
generators rebuild C and V at a displaced geometry with the same random
draws, and a central difference of the oracle energy over that displacement
gives -F exactly up to O(h^2) and rounding.  This pins the chain formula,
the signs of the pair-vector bookkeeping and the generator derivatives.
"""
import dataclasses

import numpy as np

import rix_inputs as ri
from oracle.forces import forces_stress
from oracle.grad import DenseCluster
from oracle.oracle import Oracle


def _energy(s, D):
    pk = ri.generate(s, D=False)
    o = Oracle(s)
    o.set_data(pk.C, pk.V, D)
    o.kpattern()
    return o.energy(o.build_K())


def _adjoint_dense(s, pk):
    """dE/dC and dE/dV of every stored entry from the dense definition (cluster)."""
    dc = DenseCluster(s, pk)
    dEdC = np.zeros_like(pk.C)
    dEdV = np.zeros_like(pk.V)
    nb = s.nbas[s.species]
    na = s.naux[s.species]
    for p in range(pk.n_pairs):
        a, b = pk.A[p], pk.B[p]
        rows = na[a] + (0 if pk.onsite[p] else na[b])
        for r in range(rows):
            M = dc.M_matrix(int(dc.ao[a] + r if r < na[a] else dc.ao[b] + (r - na[a])))
            blk = -0.5 * dc.D[dc.bo[a]:dc.bo[a + 1], :] @ M @ dc.D[:, dc.bo[b]:dc.bo[b + 1]]
            base = pk.offC[p] + r * nb[a] * nb[b]
            dEdC[base:base + nb[a] * nb[b]] = blk.ravel()
        for P in range(na[a]):
            CP = dc.C_matrix(int(dc.ao[a] + P))
            DCD = dc.D @ CP @ dc.D
            for Q in range(na[b]):
                CQ = dc.C_matrix(int(dc.ao[b] + Q))
                dEdV[pk.offV[p] + P * na[b] + Q] = -0.25 * float(np.sum(DCD * CQ.T))
    return dEdC, dEdV


def test_force_chain_against_finite_differences():
    import rix_inputs.systems as S
    xyz, spc = S._waters(np.array([[0.0, 0.0, 0.0], [2.9, 0.4, -0.3]]), 7)
    nb, na = S._species_arrays(["O", "H"])
    s = S.System(name="dimer", seed=7, xyz=ri.ang2bohr(xyz), species=spc, species_names=["O", "H"], nbas=nb,
                 naux=na, sigma=S._aux_widths(7, ["O", "H"]), cell=None, cutoff=0.0, tau=0.0,
                 orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))
    pk = ri.generate(s)
    dEdC, dEdV = _adjoint_dense(s, pk)
    dC, dV = pk.gen_derivatives()
    F, stress = forces_stress(s, pk, dEdC, dEdV, dC, dV)
    assert stress is None
    assert np.abs(F.sum(axis=0)).max() < 1e-10 * np.abs(F).max()     # translation invariance
    h = 1e-4
    for atom, c in ((0, 0), (1, 2), (4, 1)):
        e = []
        for sg in (1, -1):
            x = s.xyz.copy()
            x[atom, c] += sg * h
            e.append(_energy(dataclasses.replace(s, xyz=x), pk.D))
        fd = -(e[0] - e[1]) / (2 * h)
        assert abs(fd - F[atom, c]) < 1e-6 * np.abs(F).max(), (atom, c, fd, F[atom, c])
