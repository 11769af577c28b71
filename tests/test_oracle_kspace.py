"""Pins of the oracle's Bloch sum (Eq. 3) and spin channels.

* Gamma: K(k = 0) is the dense sum over images of the image-resolved blocks,
  real; every K(k) is Hermitian (K(A,E,n) = K(E,A,-n)^T) and K(-k) = K(k)*.
* Against an explicit 2x1x1 supercell (tests/test_oracle_images.py builds its
  inputs by copying blocks): the supercell's Gamma-point matrix between copy 0
  of A and copy c of E sums the primitive images with n_x = c (mod 2), so
  K(kappa = (1/2, 0, 0)) of the primitive cell = SC[(A,0),(E,0)] - SC[(A,0),(E,1)]
  and K(0) = SC[(A,0),(E,0)] + SC[(A,0),(E,1)].
* Spin: D^up = D^dn = D/2 gives K^sigma = K(D)/2 and the closed-shell E_x;
  a fully polarised state (D^dn = 0) gives E_x = 2 E_closed(D^up).
"""
import numpy as np

import rix_inputs as ri
from oracle.kspace import bloch_sum, exchange_spin
from oracle.oracle import Oracle, exchange

from test_oracle_images import _base, _relabelled, _run


def _dense_fold(s, kk, K):
    nb = s.nbas[s.species].astype(np.int64)
    bo = np.concatenate([[0], np.cumsum(nb)])
    A, E, _ = ri.unpack_key(kk)
    out = np.zeros((bo[-1], bo[-1]))
    off = 0
    for x in range(len(kk)):
        sz = nb[A[x]] * nb[E[x]]
        out[bo[A[x]]:bo[A[x] + 1], bo[E[x]]:bo[E[x] + 1]] += K[off:off + sz].reshape(nb[A[x]], nb[E[x]])
        off += sz
    return out


def test_gamma_hermitian_and_time_reversal():
    s, pk = _base()
    kk, K, _, _ = exchange(s, pk)
    kf = np.array([[0, 0, 0], [0.25, -0.1, 0.4], [-0.25, 0.1, -0.4], [0.5, 0.5, 0.5]])
    Kk = bloch_sum(s, kk, K, kf)
    assert np.abs(Kk[0].imag).max() == 0.0
    assert np.allclose(Kk[0].real, _dense_fold(s, kk, K), rtol=0, atol=1e-14 * np.abs(K).max())
    for q in range(len(kf)):
        assert np.abs(Kk[q] - Kk[q].conj().T).max() < 1e-13 * np.abs(K).max()
    assert np.abs(Kk[2] - Kk[1].conj()).max() < 1e-13 * np.abs(K).max()
    assert np.abs(Kk[1].imag).max() > 1e-3 * np.abs(K).max()      # a nontrivial phase was applied


def test_bloch_sum_against_explicit_supercell():
    s, pk = _base()
    N = s.n_atoms
    shift = np.zeros((2 * N, 3), dtype=np.int64)
    shift[N:, 0] = 1
    atom_src = np.concatenate([np.arange(N), np.arange(N)])
    cell2 = s.cell * np.array([2, 1, 1])[:, None]
    s2, pk2, _ = _relabelled(s, pk, s.xyz[atom_src] + shift @ s.cell, cell2, atom_src, shift)
    kk, K, _, _ = exchange(s, pk)
    Kk = bloch_sum(s, kk, K, [[0, 0, 0], [0.5, 0, 0]])
    K2, _ = _run(s2, pk2)
    nb = s.nbas[s.species].astype(np.int64)
    bo = np.concatenate([[0], np.cumsum(nb)])
    sc = np.zeros((2, bo[-1], bo[-1]))                  # [c][I][L]: copy 0 of A, copy c of E
    for (a2, e2, _), blk in K2.items():
        if a2 < N:
            a, e, c = a2, e2 % N, e2 // N
            sc[c, bo[a]:bo[a + 1], bo[e]:bo[e + 1]] += blk
    scale = np.abs(sc).max()
    assert np.abs(Kk[0] - (sc[0] + sc[1])).max() < 1e-13 * scale
    assert np.abs(Kk[1] - (sc[0] - sc[1])).max() < 1e-13 * scale


def test_spin_channels():
    s = ri.config(0)
    pk = ri.generate(s)
    kk, K, E, _ = exchange(s, pk)
    _, (Ku, Kd), Es = exchange_spin(s, pk, 0.5 * pk.D, 0.5 * pk.D)
    assert np.allclose(Ku, 0.5 * K, rtol=0, atol=1e-14 * np.abs(K).max())
    assert np.array_equal(Ku, Kd)
    assert abs(Es - E) < 1e-12 * abs(E)
    Du, Dd = pk.gen_D_spin()
    _, (Ku, Kd), Es = exchange_spin(s, pk, Du, Dd)
    o = Oracle(s)
    o.set_data(pk.C, pk.V, Du)
    o.kpattern()
    e_up_closed = o.energy(o.build_K())
    _, _, Ep = exchange_spin(s, pk, Du, np.zeros_like(Du))
    assert abs(Ep - 2 * e_up_closed) < 1e-12 * abs(Ep)
    assert Es < 0 and not np.isclose(Es, E)
