"""Pins of the FP64 oracle against references other than itself.

The paper prints no numerical values of K or E_x, so every pin is
mathematical: the plain four-index definition on tiny systems, a dense chain
on the 24-atom cluster, closed forms, exact symmetries and invariances, and
special cases.  Each check is chosen so that a plausible slip in the oracle
(wrong aux block, dropped term, wrong image sign, transposed operand) fails.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from rix_inputs.blocks import coulomb_sr, pack_key
from oracle.oracle import Oracle, exchange

from brute import dense_cluster, blocks_to_dense, k_blocks, brute_periodic


def _waters_system(o_pos_ang, seed, cell_side=None, cutoff_ang=None, tau=0.0):
    xyz, spc = S._waters(np.asarray(o_pos_ang, dtype=float), seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(
        name="test", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
        nbas=nb, naux=na, sigma=S._aux_widths(seed, names),
        cell=None if cell_side is None else ri.ang2bohr(np.eye(3) * cell_side),
        cutoff=0.0 if cutoff_ang is None else ri.ang2bohr(cutoff_ang), tau=tau,
        orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _compare_blocks(s, kk, K, ref):
    got = k_blocks(s, kk, K)
    assert set(got) == set(ref), "K pattern differs from the blocks the definition reaches"
    num = sum(np.sum((got[k] - ref[k]) ** 2) for k in ref)
    den = sum(np.sum(np.asarray(ref[k]) ** 2) for k in ref)
    return np.sqrt(num / den)


@pytest.mark.parametrize("o_pos,cut", [
    ([[0, 0, 0]], None),
    ([[0, 0, 0], [2.8, 0, 0]], None),
    ([[0, 0, 0], [2.8, 0, 0], [5.6, 0, 0]], 3.5),   # cutoff removes pairs
    ([[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0]], 4.0),
])
def test_four_index_definition(o_pos, cut):
    """K from explicit (ij|kl) = sum_PQ C^P_ij V_PQ C^Q_kl, then K_il = sum (ij|kl) D_jk."""
    s = _waters_system(o_pos, seed=5, cutoff_ang=cut)
    pk = ri.generate(s)
    C3, V, D, bo, _ = dense_cluster(s, pk)
    eri = np.einsum("pij,pq,qkl->ijkl", C3, V, C3, optimize=True)
    Kd = np.einsum("ijkl,jk->il", eri, D, optimize=True)
    kk, K, E, _ = exchange(s, pk)
    assert _rel(blocks_to_dense(s, kk, K, bo), Kd) < 1e-13
    Ed = -0.25 * np.einsum("li,il->", D, Kd)
    assert abs(E - Ed) < 1e-12 * abs(Ed)


def test_dense_chain_24_atoms():
    """Dense literal T = C D, U = V T, K = U C on the (H2O)8 cluster."""
    s = ri.config(0)
    pk = ri.generate(s)
    C3, V, D, bo, _ = dense_cluster(s, pk)
    T = np.einsum("pij,jk->pik", C3, D, optimize=True)
    U = np.tensordot(V, T, axes=([0], [0]))
    Kd = np.einsum("qik,qkl->il", U, C3, optimize=True)
    kk, K, E, _ = exchange(s, pk)
    assert _rel(blocks_to_dense(s, kk, K, bo), Kd) < 1e-13
    assert abs(E - (-0.25 * np.sum(D.T * Kd))) < 1e-12 * abs(E)
    assert E < 0


@pytest.mark.parametrize("nmol,side,cut", [(2, 6.0, 4.0), (1, 4.6, 4.8)])
def test_periodic_definition(nmol, side, cut):
    """Image-resolved K(A,E,n) against the per-quadruple definition (Eq. 4).

    The second case has the atom's own periodic images inside the cutoff
    (pairs (A, A, n != 0) with two aux sets)."""
    o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])[:nmol]
    s = _waters_system(o, seed=11, cell_side=side, cutoff_ang=cut)
    pk = ri.generate(s)
    if nmol == 1:
        assert any((pk.A == pk.B) & ~pk.onsite), "case must contain self-image pairs"
    kk, K, E, _ = exchange(s, pk)
    assert _compare_blocks(s, kk, K, brute_periodic(s, pk)) < 1e-13


@pytest.mark.parametrize("term", [1, 2, 3, 4])
def test_each_term(term):
    """Each of the four terms against the definition restricted to its aux classes."""
    o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])
    s = _waters_system(o, seed=13, cell_side=6.0, cutoff_ang=4.0)
    pk = ri.generate(s)
    orc = Oracle(s)
    orc.set_data(pk.C, pk.V, pk.D)
    orc.set_terms(1 << (term - 1))
    kk = orc.kpattern()
    K = orc.build_K()
    ref = brute_periodic(s, pk, terms=1 << (term - 1))
    assert _compare_blocks(s, kk, K, ref) < 1e-13


def test_term3_is_transpose_of_term2():
    """Term 3 (P on B, Q on E) equals term 2 (P on A, Q on G) transposed with the image flipped."""
    s = ri.config(0)
    pk = ri.generate(s)
    blocks = []
    for t in (2, 3):
        orc = Oracle(s)
        orc.set_data(pk.C, pk.V, pk.D)
        orc.set_terms(1 << (t - 1))
        kk = orc.kpattern()
        blocks.append(k_blocks(s, kk, orc.build_K()))
    k2, k3 = blocks
    scale = max(np.abs(b).max() for b in k2.values())
    for (a, e, n), b in k3.items():
        partner = k2[(e, a, tuple(-v for v in n))]
        assert np.abs(b - partner.T).max() < 1e-12 * scale


def _term_blocks(s, pk, t):
    orc = Oracle(s)
    orc.set_data(pk.C, pk.V, pk.D)
    orc.set_terms(1 << (t - 1))
    kk = orc.kpattern()
    return k_blocks(s, kk, orc.build_K())


@pytest.mark.parametrize("periodic", [False, True])
def test_terms_1_and_4_are_each_symmetric(periodic):
    """Terms 1 and 4 alone satisfy K_t(A,E,n) = K_t(E,A,-n)^T (term 2 alone does not).

    The library computes terms 1 and 4 for one orientation of each block and
    restores the other through K = X + X^T; this pins that each term carries the
    symmetry by itself (self-images included in the periodic cell).
    """
    if periodic:
        o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])
        s = _waters_system(o, seed=19, cell_side=6.0, cutoff_ang=5.0)
    else:
        s = ri.config(0)
    pk = ri.generate(s)
    for t in (1, 4):
        blocks = _term_blocks(s, pk, t)
        scale = max(np.abs(b).max() for b in blocks.values())
        assert scale > 0
        for (a, e, n), b in blocks.items():
            assert np.abs(b - blocks[(e, a, tuple(-v for v in n))].T).max() < 1e-13 * scale, (t, a, e, n)
    k2 = _term_blocks(s, pk, 2)
    scale = max(np.abs(b).max() for b in k2.values())
    worst = max(np.abs(b - k2[(e, a, tuple(-v for v in n))].T).max() for (a, e, n), b in k2.items())
    assert worst > 1e-3 * scale


def test_closed_form_single_function():
    """One atom, one basis function, one aux function: K = c^2 V D, E = -c^2 V D^2 / 4."""
    s = S.System(name="x", seed=0, xyz=np.zeros((1, 3)), species=np.zeros(1, np.int32),
                 species_names=["X"], nbas=np.array([1], np.int32), naux=np.array([1], np.int32),
                 sigma=[np.array([1.0])], cell=None, cutoff=0.0, tau=0.0)
    c, v, d = 0.7, 1.3, 0.45
    orc = Oracle(s)
    orc.set_data(np.array([c]), np.array([v]), np.array([d]))
    orc.kpattern()
    K = orc.build_K()
    assert K.shape == (1,)
    assert abs(K[0] - c * c * v * d) < 1e-15
    assert abs(orc.energy(K) - (-0.25 * c * c * v * d * d)) < 1e-15


def test_closed_form_two_atoms_by_loops():
    """Two one-function atoms: every term of the sum written out by pure-Python loops."""
    s = S.System(name="x2", seed=0, xyz=np.array([[0.0, 0, 0], [1.5, 0, 0]]),
                 species=np.zeros(2, np.int32), species_names=["X"],
                 nbas=np.array([1], np.int32), naux=np.array([1], np.int32),
                 sigma=[np.array([1.0])], cell=None, cutoff=0.0, tau=0.0)
    r = np.random.default_rng(3)
    # pairs (0,0) (0,1) (1,0) (1,1); C(0,1) has rows [aux0, aux1]
    c00, c11 = r.normal(), r.normal()
    c01 = r.normal(size=2)                 # C^{P}_{01}, P = aux0, aux1
    Vm = r.normal(size=(2, 2)); Vm = Vm @ Vm.T
    Dm = r.normal(size=(2, 2)); Dm = Dm + Dm.T
    C = np.array([c00, c01[0], c01[1], c01[1], c01[0], c11])  # (1,0): rows aux1, aux0
    V = np.array([Vm[0, 0], Vm[0, 1], Vm[1, 0], Vm[1, 1]])
    D = np.array([Dm[0, 0], Dm[0, 1], Dm[1, 0], Dm[1, 1]])
    Cf = np.zeros((2, 2, 2))               # [P][i][j]
    Cf[0, 0, 0] = c00; Cf[1, 1, 1] = c11
    Cf[:, 0, 1] = c01; Cf[:, 1, 0] = c01
    Kref = np.zeros((2, 2))
    for i in range(2):
        for l in range(2):
            for j in range(2):
                for k in range(2):
                    for P in range(2):
                        for Q in range(2):
                            Kref[i, l] += Cf[P, i, j] * Vm[P, Q] * Cf[Q, k, l] * Dm[j, k]
    orc = Oracle(s)
    orc.set_data(C, V, D)
    kk = orc.kpattern()
    K = orc.build_K()
    assert _rel(K.reshape(2, 2), Kref) < 1e-14
    assert abs(orc.energy(K) + 0.25 * np.sum(Dm.T * Kref)) < 1e-13


def _full(system, pk, D=None):
    orc = Oracle(system)
    orc.set_data(pk.C, pk.V, pk.D if D is None else D)
    kk = orc.kpattern()
    K = orc.build_K()
    return kk, K, orc.energy(K), orc


def test_symmetry_and_energy_sign():
    """K(A,E,n) = K(E,A,-n)^T; E_x < 0 with an untruncated PSD V and PSD D."""
    s = ri.config(0)
    pk = ri.generate(s)
    C3, V, D, bo, _ = dense_cluster(s, pk)
    ev = np.linalg.eigvalsh(V)
    assert ev.min() > -1e-12 * ev.max()
    assert np.linalg.eigvalsh(D).min() > -1e-12
    kk, K, E, _ = _full(s, pk)
    blocks = k_blocks(s, kk, K)
    scale = max(np.abs(b).max() for b in blocks.values())
    for (a, e, n), b in blocks.items():
        assert np.abs(b - blocks[(e, a, tuple(-v for v in n))].T).max() < 1e-13 * scale
    assert E < 0


def test_symmetry_periodic():
    o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])
    s = _waters_system(o, seed=17, cell_side=6.0, cutoff_ang=5.0)
    pk = ri.generate(s)
    kk, K, E, _ = _full(s, pk)
    blocks = k_blocks(s, kk, K)
    scale = max(np.abs(b).max() for b in blocks.values())
    for (a, e, n), b in blocks.items():
        assert np.abs(b - blocks[(e, a, tuple(-v for v in n))].T).max() < 1e-13 * scale


def test_linearity_in_D():
    s = ri.config(0)
    pk = ri.generate(s)
    r = np.random.default_rng(1)
    D2 = pk.D[pk.partner].copy()  # a second symmetric-pattern D: any array of the right size
    D2 = r.normal(size=pk.D.size)
    a, b = 0.7, -1.9
    _, K1, _, _ = _full(s, pk)
    _, K2, _, _ = _full(s, pk, D2)
    _, K12, _, _ = _full(s, pk, a * pk.D + b * D2)
    assert _rel(K12, a * K1 + b * K2) < 1e-13


def test_atom_permutation_invariance():
    s = ri.config(0)
    pk = ri.generate(s)
    kk, K, E, _ = _full(s, pk)
    perm = np.random.default_rng(2).permutation(s.n_atoms)        # new atom a' = old perm[a']
    s2 = S.System(name="perm", seed=s.seed, xyz=s.xyz[perm], species=s.species[perm],
                  species_names=s.species_names, nbas=s.nbas, naux=s.naux, sigma=s.sigma,
                  cell=None, cutoff=s.cutoff, tau=s.tau)
    keys2, A2, B2, n2 = ri.pair_list(s2)
    pk2 = ri.Packed(s2, keys2, A2, B2, n2)
    old = {int(k): p for p, k in enumerate(pk.keys)}
    src = np.array([old[int(pack_key(perm[a], perm[b], n))] for a, b, n in zip(A2, B2, n2)])
    pk2.C = np.concatenate([pk.C[pk.offC[p]:pk.offC[p + 1]] for p in src])
    pk2.V = np.concatenate([pk.V[pk.offV[p]:pk.offV[p + 1]] for p in src])
    pk2.D = np.concatenate([pk.D[pk.offD[p]:pk.offD[p + 1]] for p in src])
    kk2, K2, E2, _ = _full(s2, pk2)
    b1 = k_blocks(s, kk, K)
    b2 = k_blocks(s2, kk2, K2)
    scale = max(np.abs(b).max() for b in b1.values())
    for (a, e, n), blk in b2.items():
        assert np.abs(blk - b1[(int(perm[a]), int(perm[e]), n)]).max() < 1e-12 * scale
    assert abs(E2 - E) < 1e-12 * abs(E)


def test_cluster_in_huge_box_equals_cluster():
    """The periodic code path with a box far larger than the cutoff reduces to the cluster path."""
    o = [[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0]]
    s = _waters_system(o, seed=19, cutoff_ang=4.0)
    pk = ri.generate(s)
    kk, K, E, _ = _full(s, pk)
    sb = _waters_system(o, seed=19, cutoff_ang=4.0, cell_side=200.0)
    keys_b, *_ = ri.pair_list(sb)
    assert np.array_equal(keys_b, pk.keys)
    ob = Oracle(sb)
    ob.set_data(pk.C, pk.V, pk.D)
    kkb = ob.kpattern()
    Kb = ob.build_K()
    assert np.array_equal(kkb, kk)
    assert np.array_equal(Kb, K)
    assert ob.energy(Kb) == E


def test_row_subset_matches_full_rows():
    s = ri.config(0)
    pk = ri.generate(s)
    kk, K, E, orc = _full(s, pk)
    e_full, per_row = orc.energy(K, per_row=True)
    rows = np.array([3, 0, 17])
    o2 = Oracle(s)
    o2.set_data(pk.C, pk.V, pk.D)
    kk2 = o2.kpattern(rows)
    K2 = o2.build_K()
    full = k_blocks(s, kk, K)
    sub = k_blocks(s, kk2, K2)
    for key, blk in sub.items():
        assert key[0] in rows
        assert np.array_equal(blk, full[key])
    e2, pr2 = o2.energy(K2, per_row=True)
    assert np.allclose(pr2, per_row[rows], rtol=0, atol=1e-12 * abs(e_full))
    assert abs(per_row.sum() - e_full) < 1e-12 * abs(e_full)


def test_screening_drops_blocks_as_zero():
    """tau removes whole blocks: equal to the definition with those blocks zeroed."""
    s = _waters_system([[0, 0, 0], [2.8, 0, 0], [5.6, 0, 0]], seed=23, cutoff_ang=6.0, tau=0.0)
    pk = ri.generate(s)
    amax = [np.abs(pk.C[pk.offC[p]:pk.offC[p + 1]]).max() for p in range(pk.n_pairs)]
    tau = float(np.sort(amax)[len(amax) // 4]) * 1.0000001   # drops about a quarter of C blocks
    s.tau = tau
    C0, V0, D0 = pk.C.copy(), pk.V.copy(), pk.D.copy()
    for arr, off in ((C0, pk.offC), (V0, pk.offV), (D0, pk.offD)):
        for p in range(pk.n_pairs):
            if np.abs(arr[off[p]:off[p + 1]]).max() < tau:
                arr[off[p]:off[p + 1]] = 0
    kk, K, E, _ = _full(s, pk)
    s.tau = 0.0
    pz = ri.Packed(s, pk.keys, pk.A, pk.B, pk.n)
    pz.C, pz.V, pz.D = C0, V0, D0
    C3, V, D, bo, _ = dense_cluster(s, pz)
    Kd = np.einsum("ijkl,jk->il", np.einsum("pij,pq,qkl->ijkl", C3, V, C3, optimize=True), D, optimize=True)
    assert _rel(blocks_to_dense(s, kk, K, bo), Kd) < 1e-13


@pytest.mark.parametrize("i", [0, 1, 2, 3, 4])
def test_pair_list_agrees_with_generator(i):
    s = ri.config(i)
    keys, *_ = ri.pair_list(s)
    assert np.array_equal(Oracle(s).pair_keys(), keys)


def test_coulomb_generator_limits():
    """V generator: R -> 0 series continuity, omega -> 0 gives erf(R/g1)/R, symmetry, decay."""
    sP, sQ = 0.7, 1.9
    g1 = np.sqrt(2 * (sP ** 2 + sQ ** 2))
    R = np.array([0.0, 1e-4 * g1, 0.999e-3 * g1, 1.001e-3 * g1, 0.5, 3.0])
    v = coulomb_sr(R, sP, sQ, 0.11)
    g2 = np.sqrt(g1 ** 2 + 1 / 0.11 ** 2)
    assert abs(v[0] - 2 / np.sqrt(np.pi) * (1 / g1 - 1 / g2)) < 1e-15
    from scipy.special import erf as _erf
    for Rt in (0.999e-3 * g1, 1.001e-3 * g1):      # series and closed form meet at the switch
        closed = (_erf(Rt / g1) - _erf(Rt / g2)) / Rt
        series = 2 / np.sqrt(np.pi) * ((1 / g1 - 1 / g2) - Rt ** 2 / 3 * (1 / g1 ** 3 - 1 / g2 ** 3))
        assert abs(closed - series) < 1e-11 * series
        assert abs(coulomb_sr(np.array([Rt]), sP, sQ, 0.11)[0] - series) < 1e-11 * series
    from scipy.special import erf
    w = coulomb_sr(np.array([0.5, 2.0, 7.0]), sP, sQ, 1e-7)
    assert np.allclose(w, erf(np.array([0.5, 2.0, 7.0]) / g1) / np.array([0.5, 2.0, 7.0]), rtol=1e-6)
    assert np.array_equal(coulomb_sr(R, sP, sQ, 0.11), coulomb_sr(R, sQ, sP, 0.11))
    far = coulomb_sr(np.array([10.0, 20.0, 30.0]), sP, sQ, 0.11)
    assert far[0] > far[1] > far[2] > 0


@pytest.mark.parametrize("periodic", [False, True])
def test_sampled_blocks_equal_full_rows(periodic):
    """Block-sampled mode (only listed K blocks) gives exactly the full build's blocks."""
    if periodic:
        s = _waters_system([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], seed=29, cell_side=6.0, cutoff_ang=4.5)
    else:
        s = ri.config(0)
    pk = ri.generate(s)
    kk, K, E, _ = _full(s, pk)
    full = k_blocks(s, kk, K)
    pick = np.random.default_rng(4).choice(len(kk), 12, replace=False)
    o = Oracle(s)
    o.set_data(pk.C, pk.V, pk.D)
    ks = o.kpattern_blocks(kk[pick])
    Ks = o.build_K()
    got = k_blocks(s, ks, Ks)
    assert set(got) == {k for k in full if int(ri.pack_key(k[0], k[1], np.array(k[2]))) in set(kk[pick].tolist())}
    for key, blk in got.items():
        assert np.array_equal(blk, full[key])


def test_full_range_generator_is_plain_gaussian_coulomb():
    """PBE0 kernel (omega <= 0): every generated V element is erf(R/g1)/R (R -> 0: 2/(sqrt(pi) g1)),
    the omega -> 0 limit of the HSE06 form, and it exceeds the short-range one everywhere."""
    from scipy.special import erf
    s = ri.full_range(ri.config(0))
    pk = ri.generate(s, C=False, D=False)
    hse = ri.generate(ri.config(0), C=False, D=False)
    sp = s.species
    for p in range(0, pk.n_pairs, 7):
        a, b = pk.A[p], pk.B[p]
        g1 = np.sqrt(2 * (s.sigma[sp[a]][:, None] ** 2 + s.sigma[sp[b]][None, :] ** 2))
        R = pk.dist[p]
        ref = 2 / np.sqrt(np.pi) / g1 if R == 0 else erf(R / g1) / R
        got = pk.V[pk.offV[p]:pk.offV[p + 1]].reshape(g1.shape)
        assert np.allclose(got, ref, rtol=1e-14, atol=0)
        assert (got > hse.V[hse.offV[p]:hse.offV[p + 1]].reshape(g1.shape)).all()


def test_delta_build_is_linear_in_D():
    """K(D1) + K(D2 - D1) = K(D2): what an incremental build relies on (oracle, no screening)."""
    s = ri.config(0)
    pk = ri.generate(s)
    D2 = pk.D
    Du, _ = pk.gen_D_spin()
    D1 = 0.9 * D2 + 0.1 * Du
    Ks = []
    for D in (D1, D2 - D1, D2):
        o = Oracle(s)
        o.set_data(pk.C, pk.V, D)
        o.kpattern()
        Ks.append(o.build_K())
    assert np.abs(Ks[0] + Ks[1] - Ks[2]).max() < 1e-13 * np.abs(Ks[2]).max()
