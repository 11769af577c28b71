"""Pins of the oracle's periodic-image bookkeeping that do not share its image convention.

The paper's exchange matrix is a lattice sum over images (Eq. 4): a crystal
described by a larger cell, or with its atoms shifted and wrapped back into
the cell, is the same crystal, so its image-resolved K and its energy per
cell must map onto the original ones block for block.  These tests build the
inputs of the second description by copying the first one's C, V and D
blocks under the atom and image relabelling (no regeneration), run the
oracle on both, and compare:

* an explicit 2x1x1 and 1x2x1 supercell: K((A,c1), (E,c2), n') of the
  supercell equals K(A, E, n) of the primitive cell with n = 2 n' + c2 - c1
  along the doubled axis; the supercell's Gamma fold summed over the copies
  equals the primitive Gamma fold; E_x per supercell is twice E_x per cell;
* a rigid translation that carries atoms across the cell faces (wrapped back
  by lattice vectors w_A): K'(A, E, n') = K(A, E, n' + w_A - w_E), E_x equal;
* the periodic energy against the definition -1/4 sum_{A in cell 0, l}
  D_{l i} K_{i l} evaluated from the per-quadruple K of tests/brute.py with
  the partner D blocks looked up by key here, per row atom.

A convention slip (V taken at the wrong image of a chain, the partner D block
at +n instead of -n, images summed with the wrong sign) changes one side of
each identity and not the other.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.oracle import Oracle
from brute import brute_periodic, k_blocks


def _cell_system(o_frac, cell_ang, cutoff_ang, seed):
    """Waters on fractional O sites of an orthorhombic cell (sides in A)."""
    cell = np.diag(cell_ang)
    xyz, spc = S._waters(np.asarray(o_frac) @ cell, seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(
        name="image-pin", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
        nbas=nb, naux=na, sigma=S._aux_widths(seed, names), cell=ri.ang2bohr(cell),
        cutoff=ri.ang2bohr(cutoff_ang), tau=0.0,
        orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def _base():
    s = _cell_system([[0.15, 0.20, 0.12], [0.62, 0.55, 0.58]], (6.1, 5.7, 6.6), 4.3, seed=21)
    pk = ri.generate(s)
    return s, pk


def _relabelled(s, pk, xyz, cell, atom_src, shift):
    """Packed inputs of the same crystal with new atom positions / cell.

    Atom A' of the new description is atom atom_src[A'] of the old one at
    lattice shift shift[A'] (old lattice vectors): x'_A' = x_{atom_src} + shift . a.
    A new pair (A', B', n') is old pair (a, b, m) with
    m = (n' expressed in old lattice vectors) + shift[B'] - shift[A'].
    """
    s2 = S.System(name=s.name + "'", seed=s.seed, xyz=xyz, species=s.species[atom_src],
                  species_names=s.species_names, nbas=s.nbas, naux=s.naux, sigma=s.sigma, cell=cell,
                  cutoff=s.cutoff, tau=s.tau, orbital_centres=None)
    keys, A, B, n = ri.blocks.pair_list(s2)
    pk2 = ri.blocks.Packed(s2, keys, A, B, n)
    to_old = np.rint(cell @ np.linalg.inv(s.cell)).astype(np.int64)    # new lattice vectors in old ones
    assert np.allclose(to_old @ s.cell, cell)
    m = n.astype(np.int64) @ to_old + shift[B] - shift[A]
    okey = ri.pack_key(atom_src[A], atom_src[B], m)
    src = np.searchsorted(pk.keys, okey)
    assert np.array_equal(pk.keys[np.minimum(src, len(pk.keys) - 1)], okey), "pair lists do not correspond"
    C = np.empty(pk2.offC[-1]); V = np.empty(pk2.offV[-1]); D = np.empty(pk2.offD[-1])
    for p, q in enumerate(src):
        C[pk2.offC[p]:pk2.offC[p + 1]] = pk.C[pk.offC[q]:pk.offC[q + 1]]
        V[pk2.offV[p]:pk2.offV[p + 1]] = pk.V[pk.offV[q]:pk.offV[q + 1]]
        D[pk2.offD[p]:pk2.offD[p + 1]] = pk.D[pk.offD[q]:pk.offD[q + 1]]
    pk2.C, pk2.V, pk2.D = C, V, D
    return s2, pk2, to_old


def _run(s, pk):
    o = Oracle(s)
    assert np.array_equal(o.pair_keys(), pk.keys)
    o.set_data(pk.C, pk.V, pk.D)
    kk = o.kpattern()
    K = o.build_K()
    return k_blocks(s, kk, K), o.energy(K)


def _max_rel(got, ref):
    scale = max(np.abs(b).max() for b in ref.values())
    return max(np.abs(got[k] - ref[k]).max() for k in ref) / scale


@pytest.mark.parametrize("axis", [0, 1])
def test_supercell_matches_primitive_blocks_and_gamma_fold(axis):
    s, pk = _base()
    N = s.n_atoms
    reps = np.ones(3, dtype=np.int64)
    reps[axis] = 2
    cell2 = s.cell * reps[:, None]
    shift = np.zeros((2 * N, 3), dtype=np.int64)
    shift[N:, axis] = 1
    atom_src = np.concatenate([np.arange(N), np.arange(N)])
    xyz2 = s.xyz[atom_src] + shift @ s.cell
    s2, pk2, to_old = _relabelled(s, pk, xyz2, cell2, atom_src, shift)
    assert pk2.n_pairs == 2 * pk.n_pairs
    K1, E1 = _run(s, pk)
    K2, E2 = _run(s2, pk2)
    # every supercell block is the primitive block at the matching image, and vice versa
    mapped = {}
    for (a2, e2, n2), blk in K2.items():
        m = np.asarray(n2) @ to_old + shift[e2] - shift[a2]
        key = (a2 % N, e2 % N, tuple(int(v) for v in m))
        assert key in K1, key
        if a2 < N:
            mapped[key] = blk
        else:
            assert np.allclose(blk, K1[key], rtol=0, atol=1e-13 * np.abs(K1[key]).max() + 1e-300)
    assert set(mapped) == set(K1)
    assert _max_rel(mapped, K1) < 1e-13
    # Gamma folds: the primitive fold equals the supercell fold summed over the copies of E
    fold1, fold2 = {}, {}
    for (a, e, _), b in K1.items():
        fold1[(a, e)] = fold1.get((a, e), 0) + b
    for (a2, e2, _), b in K2.items():
        if a2 < N:
            fold2[(a2, e2 % N)] = fold2.get((a2, e2 % N), 0) + b
    assert set(fold1) == set(fold2)
    assert _max_rel(fold2, fold1) < 1e-13
    assert abs(E2 - 2 * E1) < 1e-12 * abs(E1)


def test_rigid_translation_across_the_cell():
    s, pk = _base()
    N = s.n_atoms
    t = np.array([0.47, 0.33, 0.61]) @ s.cell          # moves atoms across all three faces
    frac = (s.xyz + t) @ np.linalg.inv(s.cell)
    shift = -np.floor(frac).astype(np.int64)            # wrap back into [0, 1)
    assert (shift != 0).any(axis=0).all(), "every axis must see a wrapped atom"
    xyz2 = s.xyz + t + shift @ s.cell
    s2, pk2, to_old = _relabelled(s, pk, xyz2, s.cell.copy(), np.arange(N), shift)
    K1, E1 = _run(s, pk)
    K2, E2 = _run(s2, pk2)
    assert len(K2) == len(K1)
    mapped = {}
    for (a, e, n2), blk in K2.items():
        m = tuple(int(v) for v in np.asarray(n2) + shift[e] - shift[a])
        mapped[(a, e, m)] = blk
    assert set(mapped) == set(K1)
    assert _max_rel(mapped, K1) < 1e-13
    assert abs(E2 - E1) < 1e-12 * abs(E1)


def test_periodic_energy_against_the_definition():
    """E_x = -1/4 sum over cell-0 rows of sum_{E,n} <D(E,A,-n), K(A,E,n)>, per row atom."""
    s, pk = _base()
    ref = brute_periodic(s, pk)
    nb = s.nbas[s.species]
    key2p = {int(k): p for p, k in enumerate(pk.keys)}
    e_row = np.zeros(s.n_atoms)
    for (a, e, n), blk in ref.items():
        p = key2p.get(int(ri.pack_key(e, a, -np.asarray(n))), -1)   # D between l(E, n) and i(A, 0)
        if p < 0:
            continue
        d = pk.D[pk.offD[p]:pk.offD[p + 1]].reshape(nb[e], nb[a])    # D(E,A,-n)[l][i]
        e_row[a] += -0.25 * np.sum(d.T * blk)
    o = Oracle(s)
    o.set_data(pk.C, pk.V, pk.D)
    o.kpattern()
    K = o.build_K()
    E, per_row = o.energy(K, per_row=True)
    assert np.allclose(per_row, e_row, rtol=1e-12, atol=0)
    assert abs(E - e_row.sum()) < 1e-12 * abs(E)
    # the image of the partner block matters: D(E,A,+n) in its place gives another number here
    wrong = 0.0
    for (a, e, n), blk in ref.items():
        p = key2p.get(int(ri.pack_key(e, a, np.asarray(n))), -1)
        if p >= 0:
            wrong += -0.25 * np.sum(pk.D[pk.offD[p]:pk.offD[p + 1]].reshape(nb[e], nb[a]).T * blk)
    assert abs(wrong - E) > 1e-9 * abs(E)
