"""A small system with a well-conditioned auxiliary basis for the RI-fit tests.

The workloads' aux sets (56 / 16 s-Gaussians per atom, widths log-uniform in
[0.3, 3] bohr) make each pair's Coulomb metric numerically singular; a fit
test needs a metric that is not: a few even-tempered widths per atom.
"""
import numpy as np

import rix_inputs as ri
import rix_inputs.systems as S


def even_tempered_waters(o_pos_ang, seed, cell_side=None, cutoff_ang=None):
    xyz, spc = S._waters(np.asarray(o_pos_ang, dtype=float), seed)
    names = ["O", "H"]
    nb = np.array([14, 5], dtype=np.int32)
    sigma = [0.35 * 2.2 ** np.arange(6), 0.5 * 2.2 ** np.arange(4)]
    na = np.array([len(x) for x in sigma], dtype=np.int32)
    return S.System(name="even-tempered waters", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
                    nbas=nb, naux=na, sigma=sigma,
                    cell=None if cell_side is None else ri.ang2bohr(np.eye(3) * cell_side),
                    cutoff=0.0 if cutoff_ang is None else ri.ang2bohr(cutoff_ang), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def eri_from(system, pk, C0):
    """Three-centre integrals that the exact fit maps back to C0: (ij|nu) = sum_mu V^{IJ}_{nu mu} C0^mu_ij."""
    from oracle.rifit import metric
    nb = system.nbas[system.species]
    eri = np.empty_like(C0)
    for p in range(pk.n_pairs):
        M = metric(system, pk, p)
        c = C0[pk.offC[p]:pk.offC[p + 1]].reshape(M.shape[0], nb[pk.A[p]] * nb[pk.B[p]])
        eri[pk.offC[p]:pk.offC[p + 1]] = (M @ c).ravel()
    return eri
