"""Seeded synthetic C, V and D blocks in the canonical packed layout.

Canonical layout (the interchange format both the library and the oracle
read; each side builds its own pair list and checks it against ``keys``):

* pair list: all (A, B, n1, n2, n3) with |x_B + n.cell - x_A| < cutoff
  (every pair when there is no cutoff; n = 0 for clusters), sorted
  lexicographically.  The distance of a pair is evaluated in its
  representative orientation (A < B, or A == B with n > 0
  lexicographically), so the list is exactly symmetric.
* C(A,B,n): [P][i][j], P runs over aux(A) then aux(B) (aux(A) only for the
  on-site pair A == B, n == 0); i in basis(A), j in basis(B).
  C(B,A,-n)[P'][j][i] = C(A,B,n)[P][i][j] with P' the same aux function.
* V(A,B,n): [P][Q], P in aux(A), Q in aux(B) (the image of B at n).
* D(A,B,n): [i][j].
* blocks are stored back to back in pair-list order.

Generators (per the workload definitions):
* C amplitude N(0,1) * exp(-0.8 r_AB) (r in bohr), drawn for representative
  pairs and mirrored; on-site blocks symmetric in (i, j).
* V_PQ = [erf(R/g1) - erf(R/g2)] / R with g1 = sqrt(2(sP^2 + sQ^2)),
  g2 = sqrt(g1^2 + 1/omega^2); series at small R (limit 2/sqrt(pi)(1/g1 - 1/g2)).
* D = 2 sum_m c_m c_m^T over localised orbitals: coefficients
  N(0,1) * exp(-r) on every basis function of the atoms within 4 A of the
  orbital centre (nearest image), normalised to unit 2-norm.
"""
import ctypes
import math
import os
import subprocess
import threading

import numpy as np
from scipy.special import erf

from . import rng
from .systems import OMEGA, ang2bohr, D_SUPPORT_ANGSTROM

_HERE = os.path.dirname(os.path.abspath(__file__))
_GEN_SRC = os.path.join(_HERE, "_gen.c")
_GEN_LIB = os.path.join(_HERE, "_build", "libgen.so")
_gen_lock = threading.Lock()
_gen = None


def build_gen(force=False):
    """Compile the C fill helper (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_GEN_LIB), exist_ok=True)
    if force or not os.path.exists(_GEN_LIB) or os.path.getmtime(_GEN_LIB) < os.path.getmtime(_GEN_SRC):
        tmp = _GEN_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _GEN_SRC, "-lm"])
        os.replace(tmp, _GEN_LIB)
    return _GEN_LIB


def _genlib():
    global _gen
    with _gen_lock:
        if _gen is None:
            lib = ctypes.CDLL(build_gen())
            P = ctypes.c_void_p
            lib.fill_C.argtypes = [ctypes.c_int64] + [P] * 9 + [ctypes.c_uint64, ctypes.c_uint64, P]
            lib.fill_V.argtypes = [ctypes.c_int64] + [P] * 9 + [ctypes.c_double, P]
            _gen = lib
    return _gen


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)

KEY_SHIFT_A = 44
KEY_SHIFT_B = 24


def pack_key(A, B, n):
    n = np.asarray(n, dtype=np.int64)
    return ((np.asarray(A, np.int64) << KEY_SHIFT_A) | (np.asarray(B, np.int64) << KEY_SHIFT_B)
            | ((n[..., 0] + 128) << 16) | ((n[..., 1] + 128) << 8) | (n[..., 2] + 128))


def unpack_key(k):
    k = np.asarray(k, dtype=np.int64)
    A = (k >> KEY_SHIFT_A) & 0xFFFFF
    B = (k >> KEY_SHIFT_B) & 0xFFFFF
    n = np.stack([((k >> 16) & 0xFF) - 128, ((k >> 8) & 0xFF) - 128, (k & 0xFF) - 128], axis=-1)
    return A.astype(np.int32), B.astype(np.int32), n.astype(np.int32)


def image_range(system):
    """Largest |n_i| that can bring two atoms within the cutoff.

    With h_i the spacing of lattice planes and w_i the spread of the atoms'
    fractional coordinates along i, a pair at image n is at least
    (|n_i| - w_i) h_i apart, so |n_i| <= floor(cutoff / h_i + w_i).
    """
    a = np.asarray(system.cell)
    vol = abs(np.linalg.det(a))
    h = np.array([vol / np.linalg.norm(np.cross(a[1], a[2])),
                  vol / np.linalg.norm(np.cross(a[2], a[0])),
                  vol / np.linalg.norm(np.cross(a[0], a[1]))])
    frac = system.xyz @ np.linalg.inv(a)
    w = frac.max(axis=0) - frac.min(axis=0)
    return np.floor(system.cutoff / h + w).astype(int)


def _is_rep(A, B, n):
    npos = (n[:, 0] > 0) | ((n[:, 0] == 0) & ((n[:, 1] > 0) | ((n[:, 1] == 0) & (n[:, 2] > 0))))
    return (A < B) | ((A == B) & npos)


def _d2(xyz, cell, A, B, n):
    """Squared distance in the exact operation order shared by all pair builders."""
    if cell is None:
        s = np.zeros((len(A), 3))
    else:
        nn = n.astype(np.float64)
        s = (nn[:, 0:1] * cell[0][None, :] + nn[:, 1:2] * cell[1][None, :]) + nn[:, 2:3] * cell[2][None, :]
    dx = (xyz[B] + s) - xyz[A]
    return (dx[:, 0] * dx[:, 0] + dx[:, 1] * dx[:, 1]) + dx[:, 2] * dx[:, 2]


def pair_distance2(system, A, B, n):
    """d^2 of each pair evaluated in its representative orientation."""
    A = np.asarray(A); B = np.asarray(B); n = np.asarray(n)
    rep = _is_rep(A, B, n) | ((A == B) & (n == 0).all(axis=1))
    Ar = np.where(rep, A, B)
    Br = np.where(rep, B, A)
    nr = np.where(rep[:, None], n, -n)
    return _d2(system.xyz, system.cell, Ar, Br, nr)


def pair_list(system):
    """Sorted canonical pair list: keys, A, B, n.

    Candidates come from a k-d tree over the periodic images (radius padded
    by 1e-9 relative); every candidate is then decided by the exact d^2 test.
    """
    from scipy.spatial import cKDTree
    nat = system.n_atoms
    if system.cell is None:
        if system.cutoff <= 0:
            A, B = np.meshgrid(np.arange(nat), np.arange(nat), indexing="ij")
            A = A.ravel(); B = B.ravel()
            n = np.zeros((len(A), 3), dtype=np.int64)
        else:
            tree = cKDTree(system.xyz)
            cand = tree.query_pairs(system.cutoff * (1 + 1e-9), output_type="ndarray")
            A = np.concatenate([cand[:, 0], cand[:, 1], np.arange(nat)])
            B = np.concatenate([cand[:, 1], cand[:, 0], np.arange(nat)])
            n = np.zeros((len(A), 3), dtype=np.int64)
            d2 = pair_distance2(system, A, B, n)
            keep = d2 < system.cutoff * system.cutoff
            A, B, n = A[keep], B[keep], n[keep]
    else:
        if system.cutoff <= 0:
            raise ValueError("periodic systems need a cutoff")
        nr = image_range(system)
        imgs = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in nr], indexing="ij"),
                        axis=-1).reshape(-1, 3)
        shift = imgs.astype(np.float64) @ system.cell
        pts = (system.xyz[None, :, :] + shift[:, None, :]).reshape(-1, 3)
        tree = cKDTree(pts)
        lists = tree.query_ball_point(system.xyz, system.cutoff * (1 + 1e-9))
        A = np.repeat(np.arange(nat), [len(l) for l in lists])
        J = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists])
        B = J % nat
        n = imgs[J // nat].astype(np.int64)
        d2 = pair_distance2(system, A, B, n)
        keep = d2 < system.cutoff * system.cutoff
        A, B, n = A[keep], B[keep], n[keep]
    keys = pack_key(A, B, n)
    keys = np.unique(keys)
    A, B, n = unpack_key(keys)
    return keys, A, B, n


def coulomb_sr(R, sP, sQ, omega):
    """Short-range (erfc-screened) Coulomb interaction of two unit s-Gaussian
    charges of widths sP, sQ at distance R (bohr); broadcasts.  omega <= 0:
    the full-range (PBE0) interaction erf(R/g1)/R."""
    g1 = np.sqrt(2.0 * (sP * sP + sQ * sQ))
    small = R < 1e-3 * g1
    Rs = np.where(small, 1.0, R)
    if omega <= 0:
        full = erf(Rs / g1) / Rs
        ser = (2.0 / math.sqrt(math.pi)) * ((1.0 / g1) - (R * R / 3.0) * (1.0 / g1 ** 3))
        return np.where(small, ser, full)
    g2 = np.sqrt(g1 * g1 + 1.0 / (omega * omega))
    full = (erf(Rs / g1) - erf(Rs / g2)) / Rs
    ser = (2.0 / math.sqrt(math.pi)) * ((1.0 / g1 - 1.0 / g2) - (R * R / 3.0) * (1.0 / g1 ** 3 - 1.0 / g2 ** 3))
    return np.where(small, ser, full)


class Packed:
    """Canonical packed C, V, D plus the pair list they are laid out on."""

    def __init__(self, system, keys, A, B, n):
        self.system = system
        self.keys, self.A, self.B, self.n = keys, A, B, n
        sp = system.species
        nbA = system.nbas[sp[A]].astype(np.int64); nbB = system.nbas[sp[B]].astype(np.int64)
        naA = system.naux[sp[A]].astype(np.int64); naB = system.naux[sp[B]].astype(np.int64)
        self.onsite = (A == B) & (n == 0).all(axis=1)
        self.sizeC = (naA + np.where(self.onsite, 0, naB)) * nbA * nbB
        self.sizeV = naA * naB
        self.sizeD = nbA * nbB
        self.offC = np.concatenate([[0], np.cumsum(self.sizeC)]).astype(np.int64)
        self.offV = np.concatenate([[0], np.cumsum(self.sizeV)]).astype(np.int64)
        self.offD = np.concatenate([[0], np.cumsum(self.sizeD)]).astype(np.int64)
        self.partner = np.searchsorted(keys, pack_key(B, A, -n))
        assert (keys[self.partner] == pack_key(B, A, -n)).all(), "pair list not symmetric"
        self.rep = _is_rep(A, B, n) | self.onsite
        self.dist = np.sqrt(pair_distance2(system, A, B, n))
        self.C = None
        self.V = None
        self.D = None

    @property
    def n_pairs(self):
        return len(self.keys)

    def _groups(self, mask):
        sp = self.system.species
        sA = sp[self.A]; sB = sp[self.B]
        idx = np.nonzero(mask)[0]
        if len(idx) == 0:
            return
        gk = (sA[idx].astype(np.int64) * 64 + sB[idx]) * 2 + self.onsite[idx]
        for g in np.unique(gk):
            sel = idx[gk == g]
            yield int(sA[sel[0]]), int(sB[sel[0]]), bool(self.onsite[sel[0]]), sel

    def _pair_sizes(self):
        s = self.system
        sp = s.species
        return (np.ascontiguousarray(s.naux[sp[self.A]], dtype=np.int32),
                np.ascontiguousarray(s.naux[sp[self.B]], dtype=np.int32),
                np.ascontiguousarray(s.nbas[sp[self.A]], dtype=np.int32),
                np.ascontiguousarray(s.nbas[sp[self.B]], dtype=np.int32))

    def gen_C(self):
        s = self.system
        C = np.empty(int(self.offC[-1]), dtype=np.float64)
        naA, naB, nbA, nbB = self._pair_sizes()
        rep = np.ascontiguousarray(self.rep, dtype=np.uint8)
        ons = np.ascontiguousarray(self.onsite, dtype=np.uint8)
        part = np.ascontiguousarray(self.partner, dtype=np.int64)
        dist = np.ascontiguousarray(self.dist, dtype=np.float64)
        offC = np.ascontiguousarray(self.offC, dtype=np.int64)
        _genlib().fill_C(self.n_pairs, _p(offC), _p(rep), _p(ons), _p(part), _p(naA), _p(naB), _p(nbA), _p(nbB),
                         _p(dist), s.seed, rng.STREAM_C, _p(C))
        self.C = C
        return C

    def gen_V(self):
        s = self.system
        V = np.empty(int(self.offV[-1]), dtype=np.float64)
        naA, naB, _, _ = self._pair_sizes()
        sig = np.ascontiguousarray(np.concatenate(s.sigma), dtype=np.float64)
        sig_off = np.concatenate([[0], np.cumsum([len(x) for x in s.sigma])]).astype(np.int64)
        sp = s.species
        sigA = np.ascontiguousarray(sig_off[sp[self.A]], dtype=np.int64)
        sigB = np.ascontiguousarray(sig_off[sp[self.B]], dtype=np.int64)
        rep = np.ascontiguousarray(self.rep, dtype=np.uint8)
        part = np.ascontiguousarray(self.partner, dtype=np.int64)
        dist = np.ascontiguousarray(self.dist, dtype=np.float64)
        offV = np.ascontiguousarray(self.offV, dtype=np.int64)
        _genlib().fill_V(self.n_pairs, _p(offV), _p(rep), _p(part), _p(naA), _p(naB), _p(sigA), _p(sigB), _p(sig),
                         _p(dist), float(getattr(s, "omega", OMEGA)), _p(V))
        self.V = V
        return V

    def pair_vectors(self):
        """r_p = x_B + n . cell - x_A of every pair in its own orientation (bohr), [n_pairs, 3]."""
        s = self.system
        r = s.xyz[self.B] - s.xyz[self.A]
        if s.cell is not None:
            r = r + self.n.astype(np.float64) @ s.cell
        return r

    def gen_derivatives(self):
        """Derivatives of the generated C and V with respect to each pair's vector r_p.

        The generators make C(A,B,n) = g exp(-0.8 |r_p|) with draws g that do not
        depend on the geometry and V_PQ = v(|r_p|; sigma_P, sigma_Q), so
          dC/dr_p = -0.8 C r_p / |r_p|,   dV/dr_p = v'(|r_p|) r_p / |r_p|,
          v'(R) = (2/sqrt(pi)) (exp(-R^2/g1^2)/g1 - exp(-R^2/g2^2)/g2) / R - v(R) / R
        (the g2 terms absent for the full-range metric), and both vanish for
        the on-site pairs (r_p = 0).  Returns (dC [3, c_elems], dV [3, v_elems])
        in the packed layouts: what a caller passes to the force/stress chain.
        """
        s = self.system
        r = self.pair_vectors()
        R = np.sqrt((r * r).sum(axis=1))
        rhat = np.where(R[:, None] > 0, r / np.where(R > 0, R, 1.0)[:, None], 0.0)
        dC = (-0.8 * np.repeat(rhat, self.sizeC, axis=0) * self.C[:, None]).T.copy()
        dV = np.zeros((3, int(self.offV[-1])))
        omega = float(getattr(s, "omega", OMEGA))
        sp = s.species
        for p in range(self.n_pairs):
            if R[p] == 0.0:
                continue
            sP = s.sigma[sp[self.A[p]]][:, None]
            sQ = s.sigma[sp[self.B[p]]][None, :]
            g1 = np.sqrt(2.0 * (sP * sP + sQ * sQ))
            Rp = R[p]
            v = self.V[self.offV[p]:self.offV[p + 1]].reshape(g1.shape)
            d = np.exp(-Rp * Rp / (g1 * g1)) / g1
            if omega > 0:
                g2 = np.sqrt(g1 * g1 + 1.0 / (omega * omega))
                d = d - np.exp(-Rp * Rp / (g2 * g2)) / g2
            dv = (2.0 / math.sqrt(math.pi)) * d / Rp - v / Rp
            dV[:, self.offV[p]:self.offV[p + 1]] = rhat[p][:, None] * dv.reshape(1, -1)
        return dC, dV

    def orbitals(self):
        """Support of each orbital: list of (atoms, image vectors, distances in bohr)."""
        s = self.system
        rmax = ang2bohr(D_SUPPORT_ANGSTROM)
        out = []
        for c in s.orbital_centres:
            d = s.xyz - s.xyz[c][None, :]
            if s.cell is None:
                img = np.zeros((s.n_atoms, 3), dtype=np.int64)
            else:
                frac = d @ np.linalg.inv(s.cell)
                img = -np.rint(frac).astype(np.int64)
                d = d + img @ s.cell
            r = np.sqrt((d * d).sum(axis=1))
            sel = np.nonzero(r <= rmax)[0]
            out.append((sel, img[sel], r[sel]))
        return out

    def gen_D(self, weights=None):
        """D = sum_m w_m c_m c_m^T over the localised orbitals (w_m = 2: closed shell).

        weights (optional, one per orbital) gives other occupations, e.g. the
        per-spin densities of a collinear spin-polarised state (w_m in {0, 1}).
        """
        s = self.system
        D = np.zeros(int(self.offD[-1]), dtype=np.float64)
        nb = s.nbas[s.species].astype(np.int64)
        dropped = 0
        for m, (atoms, img, r) in enumerate(self.orbitals()):
            nbs = nb[atoms]
            nloc = int(nbs.sum())
            c = rng.normal(s.seed, rng.STREAM_D, (m << 20) + np.arange(nloc))
            c = c * np.repeat(np.exp(-r), nbs)
            c = c / np.linalg.norm(c)
            na = len(atoms)
            X, Y = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
            keys = pack_key(atoms[X], atoms[Y], img[Y] - img[X])
            pos = np.minimum(np.searchsorted(self.keys, keys), len(self.keys) - 1)
            ok = self.keys[pos] == keys
            dropped += int((~ok).sum())
            loc = np.concatenate([[0], np.cumsum(nbs)])
            aof = np.repeat(np.arange(na), nbs)           # atom of each local function
            iof = np.arange(nloc) - loc[aof]              # index within its atom
            pr = pos[aof[:, None], aof[None, :]]
            okr = ok[aof[:, None], aof[None, :]]
            dst = self.offD[pr] + iof[:, None] * nbs[aof][None, :] + iof[None, :]
            w = 2.0 if weights is None else float(weights[m])
            if w == 0.0:
                continue
            val = w * np.outer(c, c)
            D[dst[okr]] += val[okr]
        if weights is None:
            self.D = D
            self.D_dropped = dropped
        return D

    def gen_D_spin(self):
        """Per-spin densities (D_up, D_dn) of a spin-polarised state: every orbital singly occupied
        in both channels except every fifth one, which the down channel leaves empty."""
        n = len(self.system.orbital_centres)
        up = np.ones(n)
        dn = np.where(np.arange(n) % 5 == 4, 0.0, 1.0)
        return self.gen_D(up), self.gen_D(dn)


def generate(system, C=True, V=True, D=True):
    keys, A, B, n = pair_list(system)
    pk = Packed(system, keys, A, B, n)
    if C:
        pk.gen_C()
    if V:
        pk.gen_V()
    if D:
        pk.gen_D()
    return pk
