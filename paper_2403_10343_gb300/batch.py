"""Several independent systems in one exchange context (one launch per stage).

ClusterBatch places clusters far apart; PeriodicBatch joins periodic cells
through the union of their pair lists.

Clusters placed further apart than three pair cutoffs share no pair, no
2-hop and no 3-hop block, so one context over their union computes each
cluster's K exactly as a context of its own would (the same product lists,
the same summation order) while every stage runs as one launch over all of
them, and one CUDA graph replays the whole batch.  Atoms of cluster c follow
those of cluster c-1, so the union's packed C, V, D and K are the clusters'
packed arrays back to back, and E_x of the union is the sum of theirs.

This module only arranges coordinates and offsets (host arithmetic on
numbers the caller passes in); all exchange work runs in librix.
"""
import numpy as np


class ClusterBatch:
    """Coordinates of the union and the offsets of every cluster's blocks.

    xyz_list, species_list: per cluster, [n][3] bohr and [n] species ids.
    cutoff_bohr: the pair cutoff the context will use (> 0).
    """

    def __init__(self, xyz_list, species_list, cutoff_bohr):
        if cutoff_bohr <= 0:
            raise ValueError("batching needs a pair cutoff: without one every atom pairs with every other")
        if len(xyz_list) != len(species_list) or not xyz_list:
            raise ValueError("one species array per cluster")
        gap = 3.0 * cutoff_bohr + 1.0
        xyz, shift = [], 0.0
        self.atom_offsets = [0]
        for x, sp in zip(xyz_list, species_list):
            x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
            if len(sp) != len(x):
                raise ValueError("species and coordinates differ in length")
            lo, hi = x[:, 0].min(), x[:, 0].max()
            xyz.append(x + np.array([shift - lo, 0.0, 0.0]))
            shift += (hi - lo) + gap
            self.atom_offsets.append(self.atom_offsets[-1] + len(x))
        self.xyz = np.concatenate(xyz)
        self.species = np.concatenate([np.asarray(s, dtype=np.int32) for s in species_list])
        self.cutoff_bohr = float(cutoff_bohr)

    @property
    def n_clusters(self):
        return len(self.atom_offsets) - 1

    def ranges(self, keys):
        """Block ranges [first, last) of each cluster in a sorted key list (rix_layout keys)."""
        first_atom = (np.asarray(keys, dtype=np.int64) >> 44) & 0xFFFFF
        return [(int(np.searchsorted(first_atom, self.atom_offsets[c], side="left")),
                 int(np.searchsorted(first_atom, self.atom_offsets[c + 1], side="left")))
                for c in range(self.n_clusters)]

    @staticmethod
    def element_ranges(offsets, block_ranges):
        """Element ranges of each cluster in a packed array with block offsets [n+1]."""
        off = np.asarray(offsets)
        return [(int(off[b0]), int(off[b1])) for b0, b1 in block_ranges]


class PeriodicBatch:
    """Several independent periodic cells in one exchange context.

    Cells with different lattices cannot share a cutoff pair builder, but
    every later stage of the build only follows the pair list and the image
    vectors n of its pairs.  So the batch hands the context the union of the
    cells' own pair lists (rix_system.pairs), with the atoms of cell c after
    those of cell c-1: no pair crosses two cells, every 2- and 3-hop block
    stays inside one cell with that cell's images, and each cell's K is
    computed exactly as in a context of its own while every stage is one
    launch over all cells (one CUDA graph replays the batch).  The union's
    packed arrays are the cells' packed arrays back to back; E_x of the
    union is the sum of the cells' (per cell of each).

    cells: list of (xyz [n][3] bohr, species [n], keys) with keys the cell's
    own sorted pair keys (rix_layout / rix_inputs.pair_list).  The context's
    cell_bohr only marks it periodic (use the first cell); the force/stress
    chain, which needs each atom's lattice, is not available on a batch.
    """

    def __init__(self, cells):
        if not cells:
            raise ValueError("no cells")
        xyz, sp, rows = [], [], []
        self.atom_offsets = [0]
        for x, s, keys in cells:
            x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
            s = np.asarray(s, dtype=np.int32)
            if len(s) != len(x):
                raise ValueError("species and coordinates differ in length")
            k = np.asarray(keys, dtype=np.int64)
            A = (k >> 44) & 0xFFFFF
            B = (k >> 24) & 0xFFFFF
            n = np.stack([((k >> 16) & 0xFF) - 128, ((k >> 8) & 0xFF) - 128, (k & 0xFF) - 128], axis=1)
            if len(k) and (A.max() >= len(x) or B.max() >= len(x)):
                raise ValueError("a pair key names an atom outside its cell")
            off = self.atom_offsets[-1]
            rows.append(np.concatenate([(A + off)[:, None], (B + off)[:, None], n], axis=1))
            xyz.append(x)
            sp.append(s)
            self.atom_offsets.append(off + len(x))
        self.xyz = np.concatenate(xyz)
        self.species = np.concatenate(sp)
        self.pairs = np.concatenate(rows).astype(np.int32)

    @property
    def n_cells(self):
        return len(self.atom_offsets) - 1

    def ranges(self, keys):
        """Block ranges [first, last) of each cell in a sorted key list (rix_layout keys)."""
        first_atom = (np.asarray(keys, dtype=np.int64) >> 44) & 0xFFFFF
        return [(int(np.searchsorted(first_atom, self.atom_offsets[c], side="left")),
                 int(np.searchsorted(first_atom, self.atom_offsets[c + 1], side="left")))
                for c in range(self.n_cells)]
