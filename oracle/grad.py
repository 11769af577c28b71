"""Partial derivatives of E_x for a cluster, from the four-index definition.

Test infrastructure only: the tests may import this module; the library
under test never does.

The exchange energy of a closed-shell density matrix (Eq. 4 with the
exchange matrix of Eqs. 6-7, Gamma point, no lattice images) is

    E_x = -1/4 sum_{P,Q} V_PQ Tr(D C^P D C^Q),

where C^P is the symmetric basis-by-basis matrix of aux function P (its
entries are the stored C blocks of every pair that carries P), V the aux
Coulomb matrix and D the density matrix, all restricted to the stored
pattern.  Treating every stored entry as its own variable (the entry at
position (i, j) of C^P and the one at (j, i) are different stored entries),
the partials at symmetric inputs are

    dE/dC^P_ij = -1/2 (D M^P D)_ij,   M^P = sum_Q V_PQ C^Q,
    dE/dV_PQ   = -1/4 Tr(D C^P D C^Q),
    dE/dD_jk   = -1/2 K_jk.

Here they are evaluated with dense N x N matrices (N = number of basis
functions), one aux function at a time, so clusters of a few hundred atoms
stay within memory.  Nothing is grouped into the four terms of Eq. 11, which
keeps this independent of both the oracle's term loops and the GPU adjoint.
"""
import numpy as np


class DenseCluster:
    """Dense view of a cluster's packed C, V and D (every pair image at n = 0)."""

    def __init__(self, system, packed):
        if system.cell is not None:
            raise ValueError("dense gradients are for clusters (no lattice images)")
        pk = packed
        if not (pk.n == 0).all():
            raise ValueError("cluster pair list with a lattice image")
        self.pk = pk
        sp = system.species
        self.nb = system.nbas[sp].astype(np.int64)
        self.na = system.naux[sp].astype(np.int64)
        self.bo = np.concatenate([[0], np.cumsum(self.nb)])
        self.ao = np.concatenate([[0], np.cumsum(self.na)])
        self.N = int(self.bo[-1])
        nat = len(sp)
        self.pairs_from = [[] for _ in range(nat)]  # pairs (A, B) by A
        self.pairs_to = [[] for _ in range(nat)]    # pairs (A, B) by B
        for p in range(pk.n_pairs):
            self.pairs_from[pk.A[p]].append(p)
            self.pairs_to[pk.B[p]].append(p)
        self.D = np.zeros((self.N, self.N))
        for p in range(pk.n_pairs):
            a, b = pk.A[p], pk.B[p]
            self.D[self._rows(a), self._rows(b)] = self._blk(pk.D, pk.offD, p, (self.nb[a], self.nb[b]))

    def _rows(self, a):
        return slice(int(self.bo[a]), int(self.bo[a + 1]))

    @staticmethod
    def _blk(arr, off, p, shape):
        return arr[off[p]:off[p + 1]].reshape(shape)

    def _cblock(self, p):
        """C(A,B) as [aux rows][i][j]; rows = aux(A), then aux(B) unless on-site."""
        pk = self.pk
        a, b = pk.A[p], pk.B[p]
        rows = self.na[a] + (0 if pk.onsite[p] else self.na[b])
        return self._blk(pk.C, pk.offC, p, (rows, self.nb[a], self.nb[b]))

    def aux_atom(self, P):
        x = int(np.searchsorted(self.ao, P, side="right") - 1)
        return x, int(P - self.ao[x])

    def C_matrix(self, P):
        """C^P as a dense matrix: P on atom X appears in every stored pair with X."""
        x, q = self.aux_atom(P)
        M = np.zeros((self.N, self.N))
        for p in self.pairs_from[x]:              # C(X, B): P is row q
            M[self._rows(x), self._rows(self.pk.B[p])] = self._cblock(p)[q]
        for p in self.pairs_to[x]:                # C(A, X), A != X: P is row na_A + q
            if self.pk.onsite[p]:
                continue
            a = self.pk.A[p]
            M[self._rows(a), self._rows(x)] = self._cblock(p)[self.na[a] + q]
        return M

    def M_matrix(self, P):
        """M^P = sum_Q V_PQ C^Q over every Q with a stored V(X_P, Y_Q)."""
        pk = self.pk
        x, q = self.aux_atom(P)
        M = np.zeros((self.N, self.N))
        for pv in self.pairs_from[x]:             # V(X, Y) present
            y = pk.B[pv]
            v = self._blk(pk.V, pk.offV, pv, (self.na[x], self.na[y]))[q]   # V_PQ, Q on Y
            for p in self.pairs_from[y]:          # C(Y, Z): Q rows 0..na_Y
                M[self._rows(y), self._rows(pk.B[p])] += np.tensordot(v, self._cblock(p)[:self.na[y]], 1)
            for p in self.pairs_to[y]:            # C(Z, Y), Z != Y: Q rows na_Z..
                if pk.onsite[p]:
                    continue
                z = pk.A[p]
                M[self._rows(z), self._rows(y)] += np.tensordot(v, self._cblock(p)[self.na[z]:], 1)
        return M

    def dC(self, p, r, i, j):
        """dE/dC for the stored entry C(A,B)[r][i][j] of pair p."""
        pk = self.pk
        a, b = pk.A[p], pk.B[p]
        P = self.ao[a] + r if r < self.na[a] else self.ao[b] + (r - self.na[a])
        M = self.M_matrix(int(P))
        return -0.5 * float(self.D[self.bo[a] + i, :] @ M @ self.D[:, self.bo[b] + j])

    def dV(self, p, P, Q):
        """dE/dV for the stored entry V(X,Y)[P][Q] of pair p."""
        x, y = self.pk.A[p], self.pk.B[p]
        CP = self.C_matrix(int(self.ao[x] + P))
        CQ = self.C_matrix(int(self.ao[y] + Q))
        return -0.25 * float(np.sum((self.D @ CP @ self.D) * CQ.T))

    def energy(self):
        """E_x by the same definition (sum over every stored V_PQ); small systems only."""
        pk = self.pk
        E = 0.0
        cache = {}
        for pv in range(pk.n_pairs):
            x, y = pk.A[pv], pk.B[pv]
            V = self._blk(pk.V, pk.offV, pv, (self.na[x], self.na[y]))
            for P in range(self.na[x]):
                kP = int(self.ao[x] + P)
                if kP not in cache:
                    CP = self.C_matrix(kP)
                    cache[kP] = (CP, self.D @ CP @ self.D)
                for Q in range(self.na[y]):
                    kQ = int(self.ao[y] + Q)
                    if kQ not in cache:
                        CQ = self.C_matrix(kQ)
                        cache[kQ] = (CQ, self.D @ CQ @ self.D)
                    E += V[P, Q] * np.sum(cache[kP][1] * cache[kQ][0].T)
        return -0.25 * E
