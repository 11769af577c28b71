"""Stored-entry bookkeeping for gradient tests: transpose partners of C, V and D entries.

C(A,B)[P][i][j] pairs with C(B,A)[P'][j][i] (aux rows of the two atoms
swapped), V(X,Y)[P][Q] with V(Y,X)[Q][P], D(A,B)[i][j] with D(B,A)[j][i].
"""


def partner_C(pk, s, p, e):
    """Index (absolute) of the transpose partner of C element e of pair p."""
    sp = s.species
    a, b = pk.A[p], pk.B[p]
    nbA, nbB, naA, naB = s.nbas[sp[a]], s.nbas[sp[b]], s.naux[sp[a]], s.naux[sp[b]]
    P, r = divmod(e, nbA * nbB)
    i, j = divmod(r, nbB)
    q = pk.partner[p]
    if pk.onsite[p]:
        return pk.offC[p] + (P * nbA + j) * nbB + i
    Pq = P + naB if P < naA else P - naA
    return pk.offC[q] + (Pq * nbB + j) * nbA + i


def partner_V(pk, s, p, e):
    sp = s.species
    naA, naB = s.naux[sp[pk.A[p]]], s.naux[sp[pk.B[p]]]
    P, Q = divmod(e, naB)
    return pk.offV[pk.partner[p]] + Q * naA + P


def partner_D(pk, s, p, e):
    sp = s.species
    nbA, nbB = s.nbas[sp[pk.A[p]]], s.nbas[sp[pk.B[p]]]
    i, j = divmod(e, nbB)
    return pk.offD[pk.partner[p]] + j * nbA + i


def entries(pk, s, which, n, rng):
    off = {"C": pk.offC, "V": pk.offV, "D": pk.offD}[which]
    part = {"C": partner_C, "V": partner_V, "D": partner_D}[which]
    out = []
    while len(out) < n:
        p = int(rng.integers(pk.n_pairs))
        e = int(rng.integers(off[p + 1] - off[p]))
        g = int(off[p] + e)
        out.append((g, int(part(pk, s, p, e))))
    return out
