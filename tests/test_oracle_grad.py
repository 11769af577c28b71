"""Pins of the dense-definition gradients (oracle/grad.py) on the CPU.

E_x is quadratic in C and in D and linear in V, so a central difference of
the oracle's own energy equals the derivative up to rounding for any step;
each perturbation moves an entry together with its transpose partner and is
compared with the sum of the two partials.  The dense energy must also equal
the oracle's term-by-term energy.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.oracle import exchange
from oracle.grad import DenseCluster
from partners import entries
from brute import blocks_to_dense


def _cluster(o_pos_ang, seed, cutoff_ang=None):
    xyz, spc = S._waters(np.asarray(o_pos_ang, dtype=float), seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(name="g", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
                    nbas=nb, naux=na, sigma=S._aux_widths(seed, names), cell=None,
                    cutoff=0.0 if cutoff_ang is None else ri.ang2bohr(cutoff_ang), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


CASES = {
    "two_waters": ([[0, 0, 0], [2.8, 0.4, 0]], 21, None),
    "three_waters_cut": ([[0, 0, 0], [2.8, 0, 0], [5.6, 0.3, 0]], 5, 3.5),
}


@pytest.mark.parametrize("case", list(CASES))
def test_dense_energy_matches_oracle(case):
    s = _cluster(*CASES[case])
    pk = ri.generate(s)
    _, _, E, _ = exchange(s, pk)
    Ed = DenseCluster(s, pk).energy()
    assert abs(Ed - E) <= 1e-12 * abs(E)


@pytest.mark.parametrize("case", list(CASES))
def test_dense_gradients_match_central_differences(case):
    s = _cluster(*CASES[case])
    pk = ri.generate(s)
    dc = DenseCluster(s, pk)
    rng = np.random.default_rng(3)
    h = 1e-3
    kk, K, _, _ = exchange(s, pk)
    Kd = blocks_to_dense(s, kk, K, dc.bo)   # dE/dD_jk = -1/2 K_jk

    def energy(C, V, D):
        pk2 = ri.blocks.Packed.__new__(ri.blocks.Packed)
        pk2.__dict__.update(pk.__dict__)
        pk2.C, pk2.V, pk2.D = C, V, D
        return exchange(s, pk2)[2]

    def locate(off, g):
        p = int(np.searchsorted(off, g, side="right") - 1)
        return p, int(g - off[p])

    for which in ("C", "V", "D"):
        for e1, e2 in entries(pk, s, which, 4, rng):
            arrs = {"C": pk.C.copy(), "V": pk.V.copy(), "D": pk.D.copy()}
            base = arrs[which]
            hi = base.copy(); hi[e1] += h
            if e2 != e1: hi[e2] += h
            lo = base.copy(); lo[e1] -= h
            if e2 != e1: lo[e2] -= h
            args_hi = dict(arrs); args_hi[which] = hi
            args_lo = dict(arrs); args_lo[which] = lo
            fd = (energy(args_hi["C"], args_hi["V"], args_hi["D"]) -
                  energy(args_lo["C"], args_lo["V"], args_lo["D"])) / (2 * h)
            an = 0.0
            for g in ({e1, e2}):
                if which == "C":
                    p, e = locate(pk.offC, g)
                    a, b = pk.A[p], pk.B[p]
                    nbA, nbB = dc.nb[a], dc.nb[b]
                    r, rem = divmod(e, nbA * nbB)
                    i, j = divmod(rem, nbB)
                    an += dc.dC(p, r, i, j)
                elif which == "V":
                    p, e = locate(pk.offV, g)
                    P, Q = divmod(e, dc.na[pk.B[p]])
                    an += dc.dV(p, P, Q)
                else:
                    p, e = locate(pk.offD, g)
                    i, j = divmod(e, dc.nb[pk.B[p]])
                    a, b = pk.A[p], pk.B[p]
                    an += -0.5 * Kd[dc.bo[a] + i, dc.bo[b] + j]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (which, fd, an)
