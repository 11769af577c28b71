"""FP64 GPU path against the FP64 oracle, through the C ABI.

Tolerance: the FP64 path and the oracle sum the same products in different
orders, so K agrees to rounding: relative Frobenius error <= 1e-12, and E_x
to 1e-12 relative.  Integer work (pair list, K pattern) must be bit-exact.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.oracle import Oracle, exchange

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300.rix import Exchange, RixError, RIX_ENOTSYM, RIX_ESTATE  # noqa: E402

K_TOL = 1e-12
E_TOL = 1e-12


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def run_gpu(system, pk, **kw):
    ex = Exchange.from_system(system, **kw)
    assert np.array_equal(ex.pair_keys(), pk.keys), "device pair list differs from the canonical list"
    C, V, D = _dev(pk.C), _dev(pk.V), _dev(pk.D)
    ex.set_CV(C, V)
    K = ex.build_K(D)
    E = ex.energy(D, K)
    torch.cuda.synchronize()
    return ex, ex.k_keys(), K.cpu().numpy(), E.item(), (C, V, D)


def _offsets(system, keys):
    A, E, _ = ri.unpack_key(keys)
    nb = system.nbas[system.species].astype(np.int64)
    return np.concatenate([[0], np.cumsum(nb[A] * nb[E])])


def rows_of(system, keys, K, rows):
    """Sub-vector of K holding the blocks of the given row atoms (keys sorted by row)."""
    A = ri.unpack_key(keys)[0]
    off = _offsets(system, keys)
    sel = np.isin(A, rows)
    parts = [K[off[x]:off[x + 1]] for x in np.nonzero(sel)[0]]
    return keys[sel], np.concatenate(parts)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _small_waters(o, seed, side=None, cut=None):
    xyz, spc = S._waters(np.asarray(o, float), seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(name="t", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
                    nbas=nb, naux=na, sigma=S._aux_widths(seed, names),
                    cell=None if side is None else ri.ang2bohr(np.eye(3) * side),
                    cutoff=0.0 if cut is None else ri.ang2bohr(cut), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def _mini_perovskite(seed=31, cut=6.5):
    s = S.perovskite(1, 1, 1, seed)
    s.cutoff = ri.ang2bohr(cut)
    return s


def test_config0_full():
    s = ri.config(0)
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    ex, keys, K, E, _ = run_gpu(s, pk)
    assert np.array_equal(keys, kk)
    assert rel(K, K_ref) < K_TOL
    assert abs(E - E_ref) < E_TOL * abs(E_ref)


@pytest.mark.parametrize("case", ["pbc2", "pbc_selfimage", "cluster3_cut", "single_water"])
def test_small_systems_full(case):
    if case == "pbc2":
        s = _small_waters([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, side=6.0, cut=4.0)
    elif case == "pbc_selfimage":
        s = _small_waters([[1.0, 1.2, 0.8]], 11, side=4.6, cut=4.8)
    elif case == "cluster3_cut":
        s = _small_waters([[0, 0, 0], [2.8, 0, 0], [5.6, 0, 0]], 5, cut=3.5)
    else:
        s = _small_waters([[0, 0, 0]], 3)
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    ex, keys, K, E, _ = run_gpu(s, pk)
    assert np.array_equal(keys, kk)
    assert rel(K, K_ref) < K_TOL
    assert abs(E - E_ref) < E_TOL * abs(E_ref)


def test_mixed_species_tiles():
    """Heavy species (Pb 39/140, I 32/120) exercise every tiling path of the kernels."""
    s = _mini_perovskite()
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    ex, keys, K, E, _ = run_gpu(s, pk)
    assert np.array_equal(keys, kk)
    assert rel(K, K_ref) < K_TOL
    assert abs(E - E_ref) < E_TOL * abs(E_ref)


@pytest.mark.parametrize("cfg,rows", [(1, [0, 1, 2, 93, 94, 95]), (2, [300, 301, 302])])
def test_full_size_sampled_rows(cfg, rows):
    """Full-size workloads: sampled K rows (a whole molecule each) against the oracle's rows."""
    s = ri.config(cfg)
    pk = ri.generate(s)
    ex, keys, K, E, _ = run_gpu(s, pk)
    orc = Oracle(s)
    orc.set_data(pk.C, pk.V, pk.D)
    kk_ref = orc.kpattern(rows)
    K_ref = orc.build_K()
    e_rows_ref = orc.energy(K_ref, per_row=True)[1]
    sub_keys, sub = rows_of(s, keys, K, rows)
    assert np.array_equal(sub_keys, kk_ref)
    assert rel(sub, K_ref) < K_TOL
    # per-row energies of the GPU K (host FP64 dot) against the oracle's per-row energies
    A, B, n = ri.unpack_key(pk.keys)
    kidx = {int(k): i for i, k in enumerate(keys)}
    koff = _offsets(s, keys)
    nb = s.nbas[s.species]
    for r, e_ref in zip(rows, e_rows_ref):
        e = 0.0
        scale = 0.0
        for p in np.nonzero(A == r)[0]:
            q = pk.partner[p]
            x = kidx[int(pk.keys[p])]
            kb = K[koff[x]:koff[x + 1]].reshape(nb[r], nb[B[p]])
            dq = pk.D[pk.offD[q]:pk.offD[q + 1]].reshape(nb[B[p]], nb[r])
            e += np.sum(dq.T * kb)
            scale += np.sum(np.abs(dq.T * kb))
        # a row's energy can nearly cancel; compare against the size of its terms
        assert abs(-0.25 * e - e_ref) < 1e-12 * 0.25 * scale
    # the device energy reduction against a host sum over the device K
    A3, E3, n3 = ri.unpack_key(keys)
    host_e = 0.0
    for p in range(pk.n_pairs):
        x = kidx[int(pk.keys[p])]
        q = pk.partner[p]
        kb = K[koff[x]:koff[x + 1]].reshape(nb[A[p]], nb[B[p]])
        dq = pk.D[pk.offD[q]:pk.offD[q + 1]].reshape(nb[B[p]], nb[A[p]])
        host_e += np.sum(dq.T * kb)
    assert abs(E - (-0.25 * host_e)) < 1e-12 * abs(E)


def test_deterministic_and_graph_replay():
    s = ri.config(0)
    pk = ri.generate(s)
    ex, keys, K1, E1, (C, V, D) = run_gpu(s, pk)
    K2 = ex.build_K(D)
    torch.cuda.synchronize()
    assert np.array_equal(K2.cpu().numpy(), K1), "two builds differ bitwise"
    st = torch.cuda.Stream()
    Kg = torch.empty_like(K2)
    Eg = torch.empty(1, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        ex.build_K(D, Kg)
        ex.energy(D, Kg, Eg)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(Kg.cpu().numpy(), K1)
    assert Eg.item() == E1


def test_fold_gamma_matches_host_fold():
    s = _small_waters([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, side=6.0, cut=4.0)
    pk = ri.generate(s)
    ex, keys, K, E, (C, V, D) = run_gpu(s, pk)
    Kd = ex.fold_gamma(_dev(K), s.nbasis)
    torch.cuda.synchronize()
    A, Eb, n = ri.unpack_key(keys)
    nb = s.nbas[s.species]
    bo = np.concatenate([[0], np.cumsum(nb)])
    off = _offsets(s, keys)
    ref = np.zeros((s.nbasis, s.nbasis))
    for x in range(len(keys)):
        ref[bo[A[x]]:bo[A[x] + 1], bo[Eb[x]]:bo[Eb[x] + 1]] += K[off[x]:off[x + 1]].reshape(nb[A[x]], nb[Eb[x]])
    assert np.abs(Kd.cpu().numpy() - ref).max() < 1e-13 * np.abs(ref).max()
    assert np.abs(ref - ref.T).max() < 1e-12 * np.abs(ref).max()


def test_status_codes():
    s = ri.config(0)
    pk = ri.generate(s)
    ex = Exchange.from_system(s)
    D = _dev(pk.D)
    with pytest.raises(RixError) as e:
        ex.build_K(D)
    assert e.value.status == RIX_ESTATE
    C = pk.C.copy()
    C[pk.offC[5] + 3] += 1e-3          # breaks C(A,B) = C(B,A)^T for one pair
    with pytest.raises(RixError) as e:
        ex.set_CV(_dev(C), _dev(pk.V))
    assert e.value.status == RIX_ENOTSYM
    with pytest.raises(RixError):
        Exchange(np.zeros((0, 3)), np.zeros(0, np.int32), [5], [16])


def test_pair_lists_of_all_workloads():
    for cfg in (0, 1, 2):
        s = ri.config(cfg)
        keys, *_ = ri.pair_list(s)
        ex = Exchange.from_system(s)
        assert np.array_equal(ex.pair_keys(), keys)
        if cfg < 2:
            assert np.array_equal(ex.k_keys(), Oracle(s).kpattern())
        ex.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["cluster24", "pbc2"])
def test_row_blocks_by_atom_count(case, precision):
    """Row blocks of at most N atoms (the manual block size): results are unchanged, in mixed
    precision with the tensor-core problems split by block."""
    if case == "cluster24":
        s = ri.config(0)
    else:
        s = _small_waters([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, side=6.0, cut=4.0)
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    ktol, etol = (K_TOL, E_TOL * abs(E_ref)) if precision == "fp64" else (1e-8, 1e-6)
    for nb_atoms in (5, 2):
        ex, keys, K, E, _ = run_gpu(s, pk, block_atoms=nb_atoms, precision=precision)
        assert ex.stats()["n_row_blocks"] == -(-s.n_atoms // nb_atoms)
        assert np.array_equal(keys, kk)
        assert rel(K, K_ref) < ktol
        assert abs(E - E_ref) < etol
        ex.close()


@pytest.mark.parametrize("case", ["cluster24", "pbc2"])
def test_row_blocked_memory_plan(case):
    """A workspace too small for T and Z forces the build into row blocks; results are unchanged."""
    precision = "fp64"
    if case == "cluster24":
        s = ri.config(0)
    else:
        s = _small_waters([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, side=6.0, cut=4.0)
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    full = Exchange.from_system(s, precision=precision)
    w0, tz = full.stats()["workspace_bytes"], full.stats()["tz_bytes"]
    assert full.stats()["n_row_blocks"] == 1
    full.close()
    ktol, etol = (K_TOL, E_TOL * abs(E_ref)) if precision == "fp64" else (1e-8, 1e-6)
    seen, why = set(), []
    for frac in (0.2, 0.35, 0.5, 0.65, 0.8):   # take that share of the T and Z buffers away
        try:
            ex, keys, K, E, _ = run_gpu(s, pk, max_workspace_bytes=int(w0 - frac * tz), precision=precision)
        except RixError as err:
            why.append(str(err))
            continue
        nb = ex.stats()["n_row_blocks"]
        seen.add(nb)
        assert np.array_equal(keys, kk)
        assert rel(K, K_ref) < ktol
        assert abs(E - E_ref) < etol
        ex.close()
    assert seen and max(seen) >= 2, (seen, w0, tz, why)


def test_set_CV_from_host_arrays():
    """rix_set_CV takes host arrays as well as device buffers; K is identical."""
    s = ri.config(0)
    pk = ri.generate(s)
    ex, keys, K1, E1, (C, V, D) = run_gpu(s, pk)
    ex2 = Exchange.from_system(s)
    ex2.set_CV(np.ascontiguousarray(pk.C), np.ascontiguousarray(pk.V))
    K2 = ex2.build_K(D).cpu().numpy()
    assert np.array_equal(K1, K2)
    ex.close()
    ex2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_choice_and_cache(tmp_path, precision):
    """rix_autotune picks one of its candidate tile budgets per kernel, the build still
    matches the oracle, and a second context reads the choice back from the cache file."""
    s = _mini_perovskite()
    pk = ri.generate(s)
    kk, K_ref, E_ref, _ = exchange(s, pk)
    cache = str(tmp_path / "tiles.txt")
    ex = Exchange.from_system(s, precision=precision)
    D = _dev(pk.D)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    chosen = ex.autotune(D, cache)
    assert all(c in (4096, 8192, 12288, 16384) for c in chosen)
    K = ex.build_K(D).cpu().numpy()
    tol = K_TOL if precision == "fp64" else 1e-8
    assert rel(K, K_ref) < tol
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    ex2 = Exchange.from_system(s, precision=precision)
    ex2.set_CV(_dev(pk.C), _dev(pk.V))
    assert ex2.autotune(D, cache) == chosen
    assert open(cache).read().splitlines() == lines
    ex.close()
    ex2.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_batch_in_one_context(precision):
    """Three independent clusters in one context (one launch per stage): each cluster's K
    equals its own context's K, and E_x is the sum."""
    from paper_2403_10343_gb300.batch import ClusterBatch
    cut = 4.0
    systems = [_small_waters([[0, 0, 0], [2.8, 0.3, 0]], 5, cut=cut),
               _small_waters([[0, 0, 0]], 6, cut=cut),
               _small_waters([[0, 0, 0], [2.8, 0, 0], [0, 2.8, 0.4]], 7, cut=cut)]
    pks = [ri.generate(s) for s in systems]
    b = ClusterBatch([s.xyz for s in systems], [s.species for s in systems], ri.ang2bohr(cut))
    s0 = systems[0]
    ex = Exchange(b.xyz, b.species, s0.nbas, s0.naux, None, b.cutoff_bohr, 0.0, precision=precision)
    C = np.concatenate([p.C for p in pks])
    V = np.concatenate([p.V for p in pks])
    D = np.concatenate([p.D for p in pks])
    assert (ex.c_elems, ex.v_elems, ex.d_elems) == (C.size, V.size, D.size)
    ex.set_CV(C, V)
    Dd = _dev(D)
    K = ex.build_K(Dd).cpu().numpy()
    E = ex.energy(Dd, ex.build_K(Dd)).item()
    keys = ex.k_keys()
    nb = s0.nbas[b.species].astype(np.int64)
    A, Ek, _ = ri.unpack_key(keys)
    koff = np.concatenate([[0], np.cumsum(nb[A] * nb[Ek])])
    e_sum = 0.0
    for c, (s, pk) in enumerate(zip(systems, pks)):
        exs, keys_s, K_s, E_s, _ = run_gpu(s, pk, precision=precision)
        b0, b1 = b.ranges(keys)[c]
        assert b1 - b0 == len(keys_s)
        e0, e1 = int(koff[b0]), int(koff[b1])
        if precision == "fp64":
            assert np.array_equal(K[e0:e1], K_s)
        else:
            assert rel(K[e0:e1], K_s) < 1e-12
        e_sum += E_s
        exs.close()
    assert abs(E - e_sum) < 1e-12 * abs(e_sum)
    ex.close()


def test_caller_supplied_pair_list():
    """rix_system.pairs: the pair list of a smaller cutoff, given explicitly (shuffled) to a context
    set up with a larger cutoff, gives exactly the build of a context with the smaller cutoff, and
    the oracle's K for that cutoff."""
    o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])
    big = _small_waters(o, seed=17, side=6.0, cut=4.8)
    small = _small_waters(o, seed=17, side=6.0, cut=4.0)
    pk = ri.generate(small)
    keys, A, B, n = ri.pair_list(small)
    rows = np.concatenate([A[:, None], B[:, None], n], axis=1)
    rows = rows[np.random.default_rng(2).permutation(len(rows))]
    ex_ref, kk_ref, K_ref, E_ref, _ = run_gpu(small, pk)
    ex = Exchange.from_system(big, pairs=rows)
    assert np.array_equal(ex.pair_keys(), pk.keys)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    D = _dev(pk.D)
    K = ex.build_K(D)
    E = ex.energy(D, K).item()
    assert np.array_equal(ex.k_keys(), kk_ref)
    assert np.array_equal(K.cpu().numpy(), K_ref) and E == E_ref
    kk, Ko, Eo, _ = exchange(small, pk)
    assert rel(K.cpu().numpy(), Ko) < K_TOL
    ex.close()
    ex_ref.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_periodic_batch_equals_separate_cells(precision):
    """Two periodic cells with different lattices in one context (PeriodicBatch): each cell's K blocks
    equal its own context's (bitwise in FP64), E_x is the sum, one launch per stage for both."""
    from paper_2403_10343_gb300.batch import PeriodicBatch
    cells = [_small_waters([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]], 11, side=6.0, cut=4.5),
             _small_waters([[1.0, 1.2, 0.8]], 12, side=4.6, cut=4.8)]
    pks = [ri.generate(s) for s in cells]
    b = PeriodicBatch([(s.xyz, s.species, pk.keys) for s, pk in zip(cells, pks)])
    s0 = cells[0]
    ex = Exchange(b.xyz, b.species, s0.nbas, s0.naux, s0.cell, s0.cutoff, 0.0, precision=precision, pairs=b.pairs)
    C = np.concatenate([p.C for p in pks])
    V = np.concatenate([p.V for p in pks])
    D = np.concatenate([p.D for p in pks])
    assert (ex.c_elems, ex.v_elems, ex.d_elems) == (C.size, V.size, D.size)
    ex.set_CV(C, V)
    Dd = _dev(D)
    K = ex.build_K(Dd)
    E = ex.energy(Dd, K).item()
    K = K.cpu().numpy()
    keys = ex.k_keys()
    nb = s0.nbas[b.species].astype(np.int64)
    A, Ek, _ = ri.unpack_key(keys)
    koff = np.concatenate([[0], np.cumsum(nb[A] * nb[Ek])])
    e_sum = 0.0
    for c, (s, pk) in enumerate(zip(cells, pks)):
        exs, keys_s, K_s, E_s, _ = run_gpu(s, pk, precision=precision)
        b0, b1 = b.ranges(keys)[c]
        assert b1 - b0 == len(keys_s)
        e0, e1 = int(koff[b0]), int(koff[b1])
        if precision == "fp64":
            assert np.array_equal(K[e0:e1], K_s)
        else:
            assert rel(K[e0:e1], K_s) < 1e-12
        e_sum += E_s
        exs.close()
    assert abs(E - e_sum) < 1e-12 * abs(e_sum)
    ex.close()
