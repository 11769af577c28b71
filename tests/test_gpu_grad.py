"""Adjoint (rix_backward) against central finite differences.

E_x is quadratic in C and in D and linear in V, so a central difference
(E(x+h) - E(x-h)) / 2h equals the derivative up to rounding for any h.
Stored entries come in transpose pairs (C(A,B)[P][i][j] <-> C(B,A)[P][j][i],
V(X,Y)[P][Q] <-> V(Y,X)[Q][P], D(A,B)[i][j] <-> D(B,A)[j][i]); a perturbation
moves both partners (keeping the inputs symmetric) and is compared with the
sum of the two reported partials.
"""
import numpy as np
import pytest

import rix_inputs as ri
import rix_inputs.systems as S
from oracle.oracle import Oracle
from oracle.grad import DenseCluster
from partners import entries as _entries, partner_C as _partner_C, partner_V as _partner_V

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300.rix import Exchange, RixError  # noqa: E402
from paper_2403_10343_gb300.autograd import exchange_energy  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _small_pbc(seed=11, side=4.6, cut=4.8, nmol=1):
    o = np.array([[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]])[:nmol]
    xyz, spc = S._waters(o, seed)
    names = ["O", "H"]
    nb, na = S._species_arrays(names)
    return S.System(name="pbc", seed=seed, xyz=ri.ang2bohr(xyz), species=spc, species_names=names,
                    nbas=nb, naux=na, sigma=S._aux_widths(seed, names), cell=ri.ang2bohr(np.eye(3) * side),
                    cutoff=ri.ang2bohr(cut), tau=0.0,
                    orbital_centres=np.repeat(np.arange(0, len(spc), 3), 5).astype(np.int32))


def _fd_check(s, pk, n=12, h=1e-3, seed=0, tol=1e-7):
    ex = Exchange.from_system(s, backward=1)
    C, V, D = _dev(pk.C), _dev(pk.V), _dev(pk.D)
    ex.set_CV(C, V)
    dD, dC, dV = ex.backward(D, 1.0)
    torch.cuda.synchronize()
    grads = {"C": dC.cpu().numpy(), "V": dV.cpu().numpy(), "D": dD.cpu().numpy()}
    base = {"C": pk.C, "V": pk.V, "D": pk.D}

    def energy(arrs):
        ex.set_CV(_dev(arrs["C"]), _dev(arrs["V"]))
        Dd = _dev(arrs["D"])
        return ex.energy(Dd, ex.build_K(Dd)).item()

    rng = np.random.default_rng(seed)
    worst = 0.0
    for which in ("C", "V", "D"):
        g = grads[which]
        scale = np.abs(g).max()
        for (e1, e2) in _entries(pk, s, which, n, rng):
            arrs = {k: v.copy() for k, v in base.items()}
            arrs[which][e1] += h
            if e2 != e1:
                arrs[which][e2] += h
            ep = energy(arrs)
            arrs[which][e1] -= 2 * h
            if e2 != e1:
                arrs[which][e2] -= 2 * h
            em = energy(arrs)
            fd = (ep - em) / (2 * h)
            an = g[e1] + (g[e2] if e2 != e1 else 0.0)
            err = abs(fd - an) / scale
            worst = max(worst, err)
            assert err < tol, (which, e1, e2, fd, an, scale)
            if e2 != e1:
                assert g[e1] == g[e2], "reported partials of transpose partners differ"
    ex.close()
    return worst


def test_grad_fd_cluster24():
    s = ri.config(0)
    pk = ri.generate(s)
    _fd_check(s, pk, n=16)


def test_grad_fd_periodic_self_images():
    s = _small_pbc()
    pk = ri.generate(s)
    assert any((pk.A == pk.B) & ~pk.onsite)
    _fd_check(s, pk, n=16, seed=1)


def test_grad_fd_periodic_two_waters():
    s = _small_pbc(nmol=2, side=6.0, cut=4.0)
    pk = ri.generate(s)
    _fd_check(s, pk, n=12, seed=2)


def test_grad_fd_heavy_species():
    s = S.perovskite(1, 1, 1, 31)
    s.cutoff = ri.ang2bohr(5.0)
    pk = ri.generate(s)
    _fd_check(s, pk, n=8, seed=3)


def test_dD_is_minus_half_K_and_oracle_fd():
    """dE/dD = -K/2 entrywise; a few C and V partials against central differences of the oracle."""
    s = ri.config(0)
    pk = ri.generate(s)
    ex = Exchange.from_system(s, backward=1)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    D = _dev(pk.D)
    dD, dC, dV = ex.backward(D, 2.0)
    K = ex.build_K(D).cpu().numpy()
    torch.cuda.synchronize()
    kidx = {int(k): x for x, k in enumerate(ex.k_keys())}
    A, E, _ = ri.unpack_key(ex.k_keys())
    nb = s.nbas[s.species]
    koff = np.concatenate([[0], np.cumsum(nb[A].astype(np.int64) * nb[E])])
    dDh = dD.cpu().numpy()
    for p in range(0, pk.n_pairs, 7):
        x = kidx[int(pk.keys[p])]
        assert np.allclose(dDh[pk.offD[p]:pk.offD[p + 1]], -1.0 * K[koff[x]:koff[x + 1]], rtol=0, atol=1e-13 * np.abs(K).max())
    o = Oracle(s)
    o.kpattern()
    rng = np.random.default_rng(5)
    h = 1e-3
    for which, g, part in (("C", dC.cpu().numpy() / 2, _partner_C), ("V", dV.cpu().numpy() / 2, _partner_V)):
        for (e1, e2) in _entries(pk, s, which, 3, rng):
            arrs = {"C": pk.C.copy(), "V": pk.V.copy(), "D": pk.D}
            vals = []
            for sgn in (1, -1):
                a = {k: v.copy() for k, v in arrs.items()}
                a[which][e1] += sgn * h
                if e2 != e1:
                    a[which][e2] += sgn * h
                o.set_data(a["C"], a["V"], a["D"])
                vals.append(o.energy(o.build_K()))
            fd = (vals[0] - vals[1]) / (2 * h)
            an = g[e1] + (g[e2] if e2 != e1 else 0.0)
            assert abs(fd - an) < 1e-7 * np.abs(g).max(), (which, fd, an)


def test_autograd_function():
    s = ri.config(0)
    pk = ri.generate(s)
    ex = Exchange.from_system(s, backward=1)
    C = _dev(pk.C).requires_grad_(True)
    V = _dev(pk.V).requires_grad_(True)
    D = _dev(pk.D).requires_grad_(True)
    E = exchange_energy(D, C, V, ex)
    E.backward()
    dD, dC, dV = ex.backward(D.detach(), 1.0)
    torch.cuda.synchronize()
    assert torch.equal(D.grad, dD) and torch.equal(C.grad, dC) and torch.equal(V.grad, dV)
    assert E.item() < 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_backward_blocks_by_atom_count(precision):
    """Adjoint with row blocks of at most 5 atoms equals the single-block adjoint."""
    s = _small_pbc(seed=11, side=6.0, cut=4.0, nmol=2)
    pk = ri.generate(s)
    D = _dev(pk.D)
    out = []
    for nb_atoms in (0, 2):
        ex = Exchange.from_system(s, backward=1, precision=precision, block_atoms=nb_atoms)
        ex.set_CV(_dev(pk.C), _dev(pk.V))
        assert ex.stats()["n_row_blocks"] == (1 if nb_atoms == 0 else 3)
        out.append([x.cpu().numpy() for x in ex.backward(D, 1.0)])
        ex.close()
    tol = 1e-13 if precision == "fp64" else 1e-9
    for g, r in zip(out[1], out[0]):
        assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r)


@pytest.mark.parametrize("case", ["cluster24", "pbc2"])
def test_backward_row_blocked_plan(case):
    """A workspace too small for T and Z splits the adjoint into row blocks
    (T and Z recomputed per block); the gradients are unchanged."""
    if case == "cluster24":
        s = ri.config(0)
    else:
        s = _small_pbc(seed=11, side=6.0, cut=4.0, nmol=2)
    pk = ri.generate(s)
    D = _dev(pk.D)
    full = Exchange.from_system(s, backward=1)
    full.set_CV(_dev(pk.C), _dev(pk.V))
    assert full.stats()["n_row_blocks"] == 1
    ref = [x.cpu().numpy() for x in full.backward(D, 1.0)]
    w0, tz = full.stats()["workspace_bytes"], full.stats()["tz_bytes"]
    full.close()
    seen = set()
    for frac in (0.2, 0.35, 0.5, 0.65):   # take that share of the T and Z buffers away
        try:
            ex = Exchange.from_system(s, backward=1, max_workspace_bytes=int(w0 - frac * tz))
        except RixError:
            continue
        ex.set_CV(_dev(pk.C), _dev(pk.V))
        seen.add(ex.stats()["n_row_blocks"])
        got = [x.cpu().numpy() for x in ex.backward(D, 1.0)]
        for g, r in zip(got, ref):
            assert np.linalg.norm(g - r) <= 1e-13 * np.linalg.norm(r)
        ex.close()
    assert max(seen) >= 2, seen


def test_grad_config1_against_dense_definition():
    """(H2O)64 cluster, 192 atoms, 8 A cutoff: rix_backward partials at random
    stored C and V entries against the dense four-index definition of the
    gradient; the mixed-precision context's dD against -1/2 K of the FP64 path."""
    s = ri.config(1)
    pk = ri.generate(s)
    dc = DenseCluster(s, pk)
    D = _dev(pk.D)
    ex = Exchange.from_system(s, backward=1)
    ex.set_CV(_dev(pk.C), _dev(pk.V))
    dD, dC, dV = [x.cpu().numpy() for x in ex.backward(D, 1.0)]
    ex.close()
    rng = np.random.default_rng(7)
    got, ref = [], []
    for _ in range(16):
        p = int(rng.integers(pk.n_pairs))
        a, b = pk.A[p], pk.B[p]
        rows = dc.na[a] + (0 if pk.onsite[p] else dc.na[b])
        r, i, j = int(rng.integers(rows)), int(rng.integers(dc.nb[a])), int(rng.integers(dc.nb[b]))
        got.append(dC[pk.offC[p] + (r * dc.nb[a] + i) * dc.nb[b] + j])
        ref.append(dc.dC(p, r, i, j))
    for _ in range(16):
        p = int(rng.integers(pk.n_pairs))
        P, Q = int(rng.integers(dc.na[pk.A[p]])), int(rng.integers(dc.na[pk.B[p]]))
        got.append(dV[pk.offV[p] + P * dc.na[pk.B[p]] + Q])
        ref.append(dc.dV(p, P, Q))
    got, ref = np.array(got), np.array(ref)
    scale = np.abs(ref).max()
    print("dense-definition gradient check: max |diff| / max |ref| =", np.abs(got - ref).max() / scale)
    assert np.all(np.abs(got - ref) <= 1e-11 * np.abs(ref) + 1e-13 * scale)
    mx = Exchange.from_system(s, backward=1, precision="mixed")
    mx.set_CV(_dev(pk.C), _dev(pk.V))
    dDm = mx.backward(D, 1.0, want=("D",))[0].cpu().numpy()
    mx.close()
    assert np.linalg.norm(dD - dDm) <= 1e-8 * np.linalg.norm(dD)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_reusing_the_forward(prec):
    """rix_options.reuse_forward: rix_backward right after rix_build_K of the same D reuses the
    build's intermediates and K instead of recomputing them, with the same gradients."""
    import rix_inputs as ri
    s = ri.config(0)
    pk = ri.generate(s)
    dev = torch.device("cuda")
    C, V, D = (torch.from_numpy(x).to(dev) for x in (pk.C, pk.V, pk.D))
    out = {}
    for reuse in (0, 1):
        ex = Exchange.from_system(s, precision=prec, backward=1, reuse_forward=reuse)
        ex.set_CV(C, V)
        ex.build_K(D)
        out[reuse] = [g.cpu().numpy() for g in ex.backward(D, 1.0)]
        again = [g.cpu().numpy() for g in ex.backward(D, 1.0)]   # nothing left to reuse: recomputed
        for a, b in zip(out[reuse], again):
            assert np.abs(a - b).max() <= (0 if prec == "fp64" else 1e-9) * np.abs(a).max()
        ex.close()
    for a, b in zip(out[0], out[1]):
        assert np.abs(a - b).max() <= (0 if prec == "fp64" else 1e-9) * np.abs(a).max()
