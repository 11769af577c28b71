"""Several independent clusters in one exchange context (one launch per stage).

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
