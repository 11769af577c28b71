"""Force and stress chain of E_x, written out from its definition (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU baseline may use this
module; the library under test never does.

The paper's force and stress contributions of the exchange energy (Secs.
"EXX force and stress contributions", "Computation of Forces and Stress")
chain the adjoint of E_x through the geometry dependence of the RI
coefficients C and the Coulomb matrix V.  Every stored block of pair
p = (A, B, n) depends on the pair vector r_p = x_B + n . a - x_A, so

    dE/dx_X   = sum_p sum_e [dE/dC_pe dC_pe/dr_p + dE/dV_pe dV_pe/dr_p] (delta_{X,B_p} - delta_{X,A_p})
    F_X       = -dE/dx_X
    dE/deps   = sum_p (dE/dr_p) r_p^T          (homogeneous strain r_p -> (1 + eps) r_p)
    stress    = dE/deps / Omega

with D held fixed.  Plain loops over pairs and atoms.
"""
import numpy as np


def dE_dr(packed, dEdC, dEdV, dCdr, dVdr):
    """dE/dr_p [n_pairs, 3] from the adjoint and the derivatives of the stored entries."""
    pk = packed
    g = np.zeros((pk.n_pairs, 3))
    for p in range(pk.n_pairs):
        c0, c1 = pk.offC[p], pk.offC[p + 1]
        v0, v1 = pk.offV[p], pk.offV[p + 1]
        for c in range(3):
            g[p, c] = np.dot(dEdC[c0:c1], dCdr[c, c0:c1]) + np.dot(dEdV[v0:v1], dVdr[c, v0:v1])
    return g


def forces_stress(system, packed, dEdC, dEdV, dCdr, dVdr):
    """(F [n_atoms, 3], stress [3, 3] or None for a cluster)."""
    pk = packed
    g = dE_dr(pk, dEdC, dEdV, dCdr, dVdr)
    dx = np.zeros((system.n_atoms, 3))
    for p in range(pk.n_pairs):
        dx[pk.B[p]] += g[p]
        dx[pk.A[p]] -= g[p]
    if system.cell is None:
        return -dx, None
    r = pk.pair_vectors()
    omega = abs(np.linalg.det(system.cell))
    return -dx, g.T @ r / omega
