"""Pins of the oracle's RI-LVL fit (oracle/rifit.py, Eq. 8 with the metric of Eq. 10).

* Integrals built as (ij|nu) = V^{IJ} C0 are mapped back to C0 (the fit
  inverts the pair metric), to the metric's condition number times rounding.
* The residual V^{IJ} C - (ij|.) vanishes to rounding for arbitrary integrals.
* A pair and its partner (J, I, -n) give the same coefficients with (i, j)
  and the aux sets swapped (the partner's metric is the permuted one), and an
  on-site block is symmetric in (i, j) when its integrals are.
* The on-site metric is the on-site V block alone (aux(I) once), and the
  Tikhonov shift lambda adds lambda to every diagonal element.
"""
import numpy as np

import rix_inputs as ri
from oracle.rifit import fit_C, metric

from rifit_systems import eri_from, even_tempered_waters


def _sys(periodic):
    o = [[0.0, 0.0, 0.0], [2.9, 0.4, -0.3]] if not periodic else [[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]]
    return even_tempered_waters(o, 23, cell_side=6.0 if periodic else None, cutoff_ang=4.5 if periodic else None)


def test_fit_inverts_the_metric():
    for periodic in (False, True):
        s = _sys(periodic)
        pk = ri.generate(s)
        conds = [np.linalg.cond(metric(s, pk, p)) for p in range(pk.n_pairs)]
        eri = eri_from(s, pk, pk.C)
        C = fit_C(s, pk, eri)
        err = np.abs(C - pk.C).max() / np.abs(pk.C).max()
        assert err < 100 * max(conds) * 2.0 ** -52, (err, max(conds))


def test_residual_partner_symmetry_and_onsite():
    s = _sys(True)
    pk = ri.generate(s)
    rng = np.random.default_rng(3)
    eri = eri_from(s, pk, pk.C) + 1e-3 * np.abs(pk.C).max() * rng.normal(size=pk.C.size)
    # keep the integrals pair-symmetric, as real ones are: mirror representative pairs onto partners
    nb = s.nbas[s.species]
    na = s.naux[s.species]
    for p in range(pk.n_pairs):
        q = pk.partner[p]
        if q <= p or pk.onsite[p]:
            continue
        a, b = pk.A[p], pk.B[p]
        x = eri[pk.offC[p]:pk.offC[p + 1]].reshape(na[a] + na[b], nb[a], nb[b])
        eri[pk.offC[q]:pk.offC[q + 1]] = np.concatenate([x[na[a]:], x[:na[a]]]).transpose(0, 2, 1).ravel()
    for p in np.nonzero(pk.onsite)[0]:
        a = pk.A[p]
        x = eri[pk.offC[p]:pk.offC[p + 1]].reshape(na[a], nb[a], nb[a])
        eri[pk.offC[p]:pk.offC[p + 1]] = (0.5 * (x + x.transpose(0, 2, 1))).ravel()
    C = fit_C(s, pk, eri)
    for p in range(pk.n_pairs):
        a, b = pk.A[p], pk.B[p]
        M = metric(s, pk, p)
        c = C[pk.offC[p]:pk.offC[p + 1]].reshape(M.shape[0], -1)
        r = eri[pk.offC[p]:pk.offC[p + 1]].reshape(M.shape[0], -1)
        assert np.abs(M @ c - r).max() < 1e-12 * np.abs(r).max()
        q = pk.partner[p]
        if pk.onsite[p]:
            x = c.reshape(na[a], nb[a], nb[a])
            assert np.abs(x - x.transpose(0, 2, 1)).max() < 1e-12 * np.abs(x).max()
            assert M.shape == (na[a], na[a])
            continue
        x = c.reshape(na[a] + na[b], nb[a], nb[b])
        y = C[pk.offC[q]:pk.offC[q + 1]].reshape(na[b] + na[a], nb[b], nb[a])
        assert np.abs(np.concatenate([x[na[a]:], x[:na[a]]]).transpose(0, 2, 1) - y).max() < 1e-11 * np.abs(x).max()
    M0, M1 = metric(s, pk, 1), metric(s, pk, 1, lam=0.25)
    assert np.allclose(M1 - M0, 0.25 * np.eye(M0.shape[0]), rtol=0, atol=1e-15)
