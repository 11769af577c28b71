"""The seeded synthetic inputs: reproducible, pair-symmetric, and D positive semidefinite.

The exchange build assumes C(B,A,-n) = C(A,B,n)^T (aux of the pair's first
atom first), V(B,A,-n) = V(A,B,n)^T and D(B,A,-n) = D(A,B,n)^T (the
translational symmetry stated after Eqs. 12a-12d); the library checks C and V
bit for bit at rix_set_CV.  These tests check the generator on the CPU.
"""
import numpy as np
import pytest

import rix_inputs as ri


def _blk(arr, off, p, shape):
    return arr[off[p]:off[p + 1]].reshape(shape)


@pytest.mark.parametrize("cfg", [0, 1])
def test_generator_is_reproducible(cfg):
    s = ri.config(cfg)
    a, b = ri.generate(s), ri.generate(s)
    assert np.array_equal(a.keys, b.keys)
    for f in ("C", "V", "D"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


def test_blocks_are_pair_symmetric():
    s = ri.config(0)
    pk = ri.generate(s)
    nb = s.nbas[s.species].astype(np.int64)
    na = s.naux[s.species].astype(np.int64)
    for p in range(pk.n_pairs):
        q = pk.partner[p]
        a, b = pk.A[p], pk.B[p]
        Dp = _blk(pk.D, pk.offD, p, (nb[a], nb[b]))
        Dq = _blk(pk.D, pk.offD, q, (nb[b], nb[a]))
        assert np.array_equal(Dp, Dq.T)
        Vp = _blk(pk.V, pk.offV, p, (na[a], na[b]))
        Vq = _blk(pk.V, pk.offV, q, (na[b], na[a]))
        assert np.array_equal(Vp, Vq.T)
        if pk.onsite[p]:
            Cp = _blk(pk.C, pk.offC, p, (na[a], nb[a], nb[a]))
            assert np.array_equal(Cp, Cp.transpose(0, 2, 1))
        else:
            Cp = _blk(pk.C, pk.offC, p, (na[a] + na[b], nb[a], nb[b]))
            Cq = _blk(pk.C, pk.offC, q, (na[b] + na[a], nb[b], nb[a]))
            # aux of the own atom first: rows of a in p are the second group of q
            assert np.array_equal(Cp[:na[a]], Cq[na[b]:].transpose(0, 2, 1))
            assert np.array_equal(Cp[na[a]:], Cq[:na[b]].transpose(0, 2, 1))


def test_density_matrix_is_positive_semidefinite():
    s = ri.config(0)
    pk = ri.generate(s)
    nb = s.nbas[s.species].astype(np.int64)
    bo = np.concatenate([[0], np.cumsum(nb)])
    N = int(bo[-1])
    D = np.zeros((N, N))
    for p in range(pk.n_pairs):
        a, b = pk.A[p], pk.B[p]
        D[bo[a]:bo[a + 1], bo[b]:bo[b + 1]] = _blk(pk.D, pk.offD, p, (nb[a], nb[b]))
    assert np.array_equal(D, D.T)
    w = np.linalg.eigvalsh(D)
    assert w.min() > -1e-12 * w.max()
    # D = 2 sum_occ c c^T with unit-norm orbitals: the trace is twice the orbital count
    n_occ = len(s.orbital_centres)
    assert abs(np.trace(D) - 2.0 * n_occ) < 1e-12 * n_occ
    assert np.sum(w > 1e-10 * w.max()) <= n_occ
