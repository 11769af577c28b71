"""Bloch sums and spin channels of the exchange matrix, written out from their definitions.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may use this module; the library under test never does.

* Bloch sum (paper Eq. 3, the Fock operator in k space):
      K_IL(k) = sum_n exp(i k . R_n) K(A,E,n)[i][l]
  with k = sum_c kappa_c b_c, R_n = sum_c n_c a_c and b_c . a_d = 2 pi delta_cd,
  so k . R_n = 2 pi kappa . n.  One explicit loop over the image-resolved
  blocks; no FFT, no blocking.
* Collinear spin (the spin index of Eqs. 3-5): the exchange matrix of each
  channel is the build with that channel's density D^sigma, and
      E_x = -1/2 sum_sigma Tr(D^sigma K^sigma),
  which for D^up = D^dn = D/2 is the closed-shell -1/4 Tr(D K).
"""
import numpy as np

import rix_inputs as ri

from .oracle import Oracle


def bloch_sum(system, kkeys, K, kfrac):
    """Dense complex K(k) [n_k, nbasis, nbasis] from packed image-resolved K blocks."""
    kf = np.asarray(kfrac, dtype=np.float64).reshape(-1, 3)
    nb = system.nbas[system.species].astype(np.int64)
    bo = np.concatenate([[0], np.cumsum(nb)])
    A, E, n = ri.unpack_key(kkeys)
    out = np.zeros((len(kf), bo[-1], bo[-1]), dtype=np.complex128)
    off = 0
    for x in range(len(kkeys)):
        a, e = int(A[x]), int(E[x])
        size = nb[a] * nb[e]
        blk = np.asarray(K[off:off + size]).reshape(nb[a], nb[e])
        off += size
        for q in range(len(kf)):
            phase = np.exp(2j * np.pi * float(np.dot(kf[q], n[x])))
            out[q, bo[a]:bo[a + 1], bo[e]:bo[e + 1]] += phase * blk
    return out


def exchange_spin(system, packed, D_up, D_dn):
    """(K keys, [K_up, K_dn], E_x) of a collinear spin-polarised density from the oracle."""
    Ks, e = [], 0.0
    kk = None
    for Ds in (D_up, D_dn):
        o = Oracle(system)
        o.set_data(packed.C, packed.V, Ds)
        kk = o.kpattern()
        K = o.build_K()
        Ks.append(K)
        # the oracle's energy is -1/4 <D, K>; a spin channel carries -1/2 <D^sigma, K^sigma>
        e += 2.0 * o.energy(K)
    return kk, Ks, e
