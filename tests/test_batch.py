"""ClusterBatch (host arithmetic): the union of clusters has exactly the clusters'
pairs, shifted by the atom offsets, so its packed arrays are theirs back to back."""
import numpy as np

import rix_inputs as ri
import rix_inputs.systems as S
from paper_2403_10343_gb300.batch import ClusterBatch


def _cluster(o, seed, cut):
    xyz, spc = S._waters(np.asarray(o, float), seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(name="c", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names, nbas=nb,
                    naux=na, sigma=S._aux_widths(seed, names), cell=None, cutoff=ri.ang2bohr(cut), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def test_union_pairs_are_the_clusters_pairs():
    cut = 4.0
    systems = [_cluster([[0, 0, 0], [2.8, 0.3, 0]], 5, cut), _cluster([[0, 0, 0]], 6, cut),
               _cluster([[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0.4]], 7, cut)]
    b = ClusterBatch([s.xyz for s in systems], [s.species for s in systems], ri.ang2bohr(cut))
    u = S.System(name="u", seed=0, xyz=b.xyz, species=b.species, species_names=systems[0].species_names,
                 nbas=systems[0].nbas, naux=systems[0].naux, sigma=systems[0].sigma, cell=None,
                 cutoff=b.cutoff_bohr, tau=0.0, orbital_centres=np.zeros(0, np.int32))
    keys_u = ri.pair_list(u)[0]
    expect = []
    for c, s in enumerate(systems):
        k, A, B, n = ri.pair_list(s)
        off = b.atom_offsets[c]
        expect.append(ri.pack_key(A + off, B + off, n))
    assert np.array_equal(keys_u, np.concatenate(expect))
    rng = b.ranges(keys_u)
    assert [r1 - r0 for r0, r1 in rng] == [len(e) for e in expect]


def test_periodic_batch_pairs_are_the_cells_pairs():
    """PeriodicBatch: the union pair list is every cell's own list with its atoms offset."""
    from paper_2403_10343_gb300.batch import PeriodicBatch
    cells = []
    for o, seed, side in (([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, 6.0), ([[1.0, 1.2, 0.8]], 12, 4.6)):
        xyz, spc = S._waters(np.asarray(o, float), seed)
        nb, na = S._species_arrays(["O", "H"])
        s = S.System(name="p", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=["O", "H"], nbas=nb,
                     naux=na, sigma=S._aux_widths(seed, ["O", "H"]), cell=ri.ang2bohr(np.eye(3) * side),
                     cutoff=ri.ang2bohr(4.5), tau=0.0, orbital_centres=np.zeros(0, np.int32))
        cells.append(s)
    b = PeriodicBatch([(s.xyz, s.species, ri.pair_list(s)[0]) for s in cells])
    expect = []
    for c, s in enumerate(cells):
        k, A, B, n = ri.pair_list(s)
        off = b.atom_offsets[c]
        expect.append(ri.pack_key(A + off, B + off, n))
    got = np.sort(ri.pack_key(b.pairs[:, 0], b.pairs[:, 1], b.pairs[:, 2:]))
    assert np.array_equal(got, np.concatenate(expect))
    assert [r1 - r0 for r0, r1 in b.ranges(got)] == [len(e) for e in expect]
