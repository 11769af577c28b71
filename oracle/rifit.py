"""RI-LVL coefficient fit written out from its definition (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU baseline may use this
module; the library under test never does.

Paper Eq. 8 with the metric of Eq. 10: for every atom pair (I, J, n)
    C^mu_ij = sum_{nu in P(IJ)} (ij|nu) L_{nu mu},   L = (V^{IJ} + lambda 1)^{-1},
P(IJ) = aux(I) then aux(J) (aux(I) alone for the on-site pair), V^{IJ} the
Coulomb matrix on P(IJ) from the blocks V(I,I,0), V(I,J,n), V(J,J,0).  One
pair at a time: assemble the metric, factor it (numpy Cholesky) and solve
(scipy triangular solves) -- library routines as the steps, no batching.
lambda = 0 is the plain inverse of the paper; lambda > 0 a Tikhonov shift.
"""
import numpy as np
from scipy.linalg import solve_triangular

import rix_inputs as ri


def metric(system, packed, p, lam=0.0):
    """V^{IJ} + lam 1 of pair p."""
    pk = packed
    na = system.naux[system.species]
    a, b = int(pk.A[p]), int(pk.B[p])
    key = {int(k): q for q, k in enumerate(pk.keys)}

    def blk(q, r, c):
        return pk.V[pk.offV[q]:pk.offV[q + 1]].reshape(r, c)

    Vaa = blk(key[int(ri.pack_key(a, a, np.zeros(3, int)))], na[a], na[a])
    if pk.onsite[p]:
        M = Vaa.copy()
    else:
        Vbb = blk(key[int(ri.pack_key(b, b, np.zeros(3, int)))], na[b], na[b])
        Vab = blk(p, na[a], na[b])
        M = np.block([[Vaa, Vab], [Vab.T, Vbb]])
    return M + lam * np.eye(M.shape[0])


def fit_C(system, packed, eri, lam=0.0):
    """Packed C fitted from the packed three-centre integrals eri (same layout as C)."""
    pk = packed
    nb = system.nbas[system.species]
    C = np.empty_like(eri)
    for p in range(pk.n_pairs):
        a, b = int(pk.A[p]), int(pk.B[p])
        M = metric(system, pk, p, lam)
        L = np.linalg.cholesky(M)
        rhs = eri[pk.offC[p]:pk.offC[p + 1]].reshape(M.shape[0], nb[a] * nb[b])
        y = solve_triangular(L, rhs, lower=True)
        C[pk.offC[p]:pk.offC[p + 1]] = solve_triangular(L.T, y, lower=False).ravel()
    return C
