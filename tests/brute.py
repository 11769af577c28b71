"""Independent references for pinning the oracle (test helpers).

* ``dense_cluster``: dense three-index C, dense V and D of a cluster (all
  blocks at n = 0), for the plain four-index definition
  K_il = sum_{jkPQ} C^P_ij V_PQ C^Q_kl D_jk.
* ``brute_periodic``: K(A,E,n) of every cell-0 row atom straight from the
  definition, one node quadruple (A, B', G', E') at a time, with the aux sets
  P in aux(A) u aux(B') and Q in aux(G') u aux(E') and V looked up per node
  pair -- no grouping into terms.
"""
import numpy as np

import rix_inputs as ri


def dense_cluster(system, pk):
    s = system
    sp = s.species
    nb = s.nbas[sp]
    na = s.naux[sp]
    bo = np.concatenate([[0], np.cumsum(nb)])
    ao = np.concatenate([[0], np.cumsum(na)])
    N, M = bo[-1], ao[-1]
    C3 = np.zeros((M, N, N))
    V = np.zeros((M, M))
    D = np.zeros((N, N))
    for p in range(pk.n_pairs):
        A, B = pk.A[p], pk.B[p]
        assert (pk.n[p] == 0).all()
        c = pk.C[pk.offC[p]:pk.offC[p + 1]]
        if pk.onsite[p]:
            C3[ao[A]:ao[A + 1], bo[A]:bo[A + 1], bo[B]:bo[B + 1]] = c.reshape(na[A], nb[A], nb[B])
        else:
            c = c.reshape(na[A] + na[B], nb[A], nb[B])
            C3[ao[A]:ao[A + 1], bo[A]:bo[A + 1], bo[B]:bo[B + 1]] = c[:na[A]]
            C3[ao[B]:ao[B + 1], bo[A]:bo[A + 1], bo[B]:bo[B + 1]] = c[na[A]:]
        V[ao[A]:ao[A + 1], ao[B]:ao[B + 1]] = pk.V[pk.offV[p]:pk.offV[p + 1]].reshape(na[A], na[B])
        D[bo[A]:bo[A + 1], bo[B]:bo[B + 1]] = pk.D[pk.offD[p]:pk.offD[p + 1]].reshape(nb[A], nb[B])
    return C3, V, D, bo, ao


def blocks_to_dense(system, kkeys, K, bo):
    """Scatter K blocks (all at n = 0) into a dense matrix."""
    A, E, n = ri.unpack_key(kkeys)
    assert (n == 0).all()
    nb = system.nbas[system.species]
    off = np.concatenate([[0], np.cumsum(nb[A] * nb[E])])
    out = np.zeros((bo[-1], bo[-1]))
    for x in range(len(kkeys)):
        out[bo[A[x]]:bo[A[x] + 1], bo[E[x]]:bo[E[x] + 1]] = K[off[x]:off[x + 1]].reshape(nb[A[x]], nb[E[x]])
    return out


def k_blocks(system, kkeys, K):
    """dict (A, E, n-tuple) -> block."""
    A, E, n = ri.unpack_key(kkeys)
    nb = system.nbas[system.species]
    off = np.concatenate([[0], np.cumsum(nb[A] * nb[E])])
    return {(int(A[x]), int(E[x]), tuple(int(v) for v in n[x])):
            K[off[x]:off[x + 1]].reshape(nb[A[x]], nb[E[x]]) for x in range(len(kkeys))}


def brute_periodic(s, pk, terms=15):
    """K blocks of the cell-0 rows from the definition, quadruple by quadruple.

    ``terms`` restricts the aux classes (bit 0: P on A, Q on E; bit 1: P on A,
    Q on G'; bit 2: P on B', Q on E'; bit 3: P on B', Q on G') for per-term pins.
    """
    sp = s.species
    nb = s.nbas[sp]
    na = s.naux[sp]
    key2p = {int(k): p for p, k in enumerate(pk.keys)}
    nbr = {}
    for p in range(pk.n_pairs):
        nbr.setdefault(int(pk.A[p]), []).append(p)

    def blk(arr, off, p, shape):
        return arr[off[p]:off[p + 1]].reshape(shape)

    def pid(a, b, m):
        return key2p.get(int(ri.pack_key(a, b, np.asarray(m))), -1)

    K = {}
    for A in range(s.n_atoms):
        for p1 in nbr[A]:
            B = int(pk.B[p1]); n1 = pk.n[p1].astype(int)
            c1 = blk(pk.C, pk.offC, p1, (-1, nb[A], nb[B]))
            Pset = [(A, np.zeros(3, int), c1[:na[A]], 0)]
            if not pk.onsite[p1]:
                Pset.append((B, n1, c1[na[A]:], 1))
            for p2 in nbr[B]:
                G = int(pk.B[p2]); n2 = n1 + pk.n[p2]
                Dbg = blk(pk.D, pk.offD, p2, (nb[B], nb[G]))
                for p3 in nbr[G]:
                    E = int(pk.B[p3]); n3 = n2 + pk.n[p3]
                    c3 = blk(pk.C, pk.offC, p3, (-1, nb[G], nb[E]))
                    # Q on E' is the first class (term 1/3), Q on G' != E' the second
                    Qset = [(E, n3, c3[na[G]:] if not pk.onsite[p3] else c3[:na[G]], 0)]
                    if not pk.onsite[p3]:
                        Qset.append((G, n2, c3[:na[G]], 1))
                    acc = np.zeros((nb[A], nb[E]))
                    for (X, nx, cP, pcls) in Pset:
                        for (Y, ny, cQ, qcls) in Qset:
                            if not (terms >> (2 * pcls + qcls)) & 1:
                                continue
                            pv = pid(X, Y, ny - nx)
                            if pv < 0:
                                continue
                            v = blk(pk.V, pk.offV, pv, (na[X], na[Y]))
                            # (ij|kl) = sum_PQ cP[P,i,j] v[P,Q] cQ[Q,k,l]
                            w = v @ cQ.reshape(cQ.shape[0], -1)            # [P, k l]
                            eri = cP.reshape(cP.shape[0], -1).T @ w          # [i j, k l]
                            eri = eri.reshape(nb[A], nb[B], nb[G], nb[E])
                            acc += np.tensordot(eri, Dbg, axes=([1, 2], [0, 1]))
                    key = (A, E, tuple(int(v) for v in n3))
                    K[key] = K.get(key, 0) + acc
    return K
