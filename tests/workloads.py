"""Helpers for checking full-size workloads against the oracle on sampled K blocks and rows."""
import numpy as np

import rix_inputs as ri


def k_offsets(s, keys):
    """Element offsets of the packed K blocks with the given (sorted) keys."""
    A, E, _ = ri.unpack_key(keys)
    nb = s.nbas[s.species].astype(np.int64)
    return np.concatenate([[0], np.cumsum(nb[A] * nb[E])])


def sample_keys(s, keys, rng, per_species=2, per_row=6):
    """A few K blocks of a few row atoms of every species (always the diagonal block)."""
    A, E, n = ri.unpack_key(keys)
    pick = []
    for sp in range(len(s.nbas)):
        atoms = np.nonzero(s.species == sp)[0]
        if len(atoms) == 0:
            continue
        for a in rng.choice(atoms, min(per_species, len(atoms)), replace=False):
            rows = np.nonzero(A == a)[0]
            diag = rows[(E[rows] == a) & (n[rows] == 0).all(axis=1)]
            pick += list(diag) + list(rng.choice(rows, min(per_row, len(rows)), replace=False))
    return np.unique(keys[np.array(pick)])


def gather_blocks(keys_all, off, K, want):
    """The blocks `want` (sorted keys) of a packed K, concatenated."""
    idx = np.searchsorted(keys_all, want)
    assert np.array_equal(keys_all[idx], want)
    return np.concatenate([np.asarray(K[off[x]:off[x + 1]]) for x in idx])


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rows_of(s, keys, K, rows):
    """Keys and concatenated blocks of the given row atoms (keys sorted by row)."""
    A = ri.unpack_key(keys)[0]
    off = k_offsets(s, keys)
    sel = np.nonzero(np.isin(A, rows))[0]
    return keys[sel], np.concatenate([np.asarray(K[off[x]:off[x + 1]]) for x in sel])


def row_energies(s, pk, keys, K, rows):
    """-1/4 sum over the pairs (r, B, n) of <D(B, r, -n), K(r, B, n)> for each row atom r, and the
    sum of the absolute terms (the scale a row's energy is compared against)."""
    A, B, _ = ri.unpack_key(pk.keys)
    kidx = {int(k): i for i, k in enumerate(keys)}
    off = k_offsets(s, keys)
    nb = s.nbas[s.species]
    out, scale = [], []
    for r in rows:
        e = a = 0.0
        for p in np.nonzero(A == r)[0]:
            q = pk.partner[p]
            x = kidx[int(pk.keys[p])]
            kb = np.asarray(K[off[x]:off[x + 1]]).reshape(nb[r], nb[B[p]])
            dq = pk.D[pk.offD[q]:pk.offD[q + 1]].reshape(nb[B[p]], nb[r])
            e += float(np.sum(dq.T * kb))
            a += float(np.sum(np.abs(dq.T * kb)))
        out.append(-0.25 * e)
        scale.append(0.25 * a)
    return np.array(out), np.array(scale)
