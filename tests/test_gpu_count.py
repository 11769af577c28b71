"""rix_count_flops: the FLOPs of a build after block screening.

The T, U2 and Z counts are checked against a count taken here from the pair
list alone (Eq. 12 products: T(A,G') <- C(A,B') D(B',G'), U2(A,G') <- V(A,G')
T(A,G'), Z(B,E') <- D(B,G') V(B,G') C(G',E') with (G',E') not on-site), with
the screening test of Sec. "Screening" (a block is kept when its largest
magnitude is >= tau) applied to the generated C, V and D.  Without screening
every count equals the setup-time count of rix_stats.
"""
import numpy as np
import pytest

import rix_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300.rix import Exchange  # noqa: E402


def _keep(arr, off, tau):
    n = len(off) - 1
    if tau <= 0:
        return np.ones(n, bool)
    return np.array([np.abs(arr[off[p]:off[p + 1]]).max(initial=0.0) >= tau for p in range(n)])


def host_counts(s, pk, D):
    nb = s.nbas[s.species].astype(np.float64)
    na = s.naux[s.species].astype(np.float64)
    A, B = pk.A, pk.B
    kC, kV, kD = _keep(pk.C, pk.offC, s.tau), _keep(pk.V, pk.offV, s.tau), _keep(D, pk.offD, s.tau)
    nat = len(s.species)
    # per atom b: sum over kept D(b, G') of nb_G; sum over kept, not on-site C(b, E') of nb_E
    sD = np.bincount(A, weights=kD * nb[B], minlength=nat)
    sC = np.bincount(A, weights=(kC & ~pk.onsite) * nb[B], minlength=nat)
    T = float(np.sum(kC * 2.0 * na[A] * nb[A] * nb[B] * sD[B]))
    U2 = float(np.sum(kV * 2.0 * na[A] * na[B] * nb[A] * nb[B]))
    Z = float(np.sum((kD & kV) * 2.0 * na[A] * nb[B] * (na[B] + nb[A]) * sC[B]))
    return T, U2, Z


@pytest.mark.parametrize("cfg", [0, 1])
def test_count_flops_fp64(cfg):
    s = ri.config(cfg)
    pk = ri.generate(s)
    ex = Exchange.from_system(s, precision="fp64")
    ex.set_CV(pk.C, pk.V)
    D = torch.from_numpy(pk.D).cuda()
    c = ex.count_flops(D)
    st = ex.stats()
    T, U2, Z = host_counts(s, pk, pk.D)
    assert c["T"] == T and c["U2"] == U2 and c["Z"] == Z
    assert c["sym"] == st["flops_stage"][5]
    assert c["term1_tc"] == c["z_tc"] == c["t_tc"] == 0.0
    for i, k in enumerate(("T", "U2", "X12", "Z", "X34")):
        assert 0 < c[k] <= st["flops_stage"][i]
        if s.tau <= 0:
            assert c[k] == st["flops_stage"][i], k
    assert c["term2"] <= st["flops_term2"]
    # a zero density: every product through D is screened out; X12 and X34 do not read D
    c0 = ex.count_flops(torch.zeros_like(D))
    if s.tau > 0:
        assert c0["T"] == 0.0 and c0["Z"] == 0.0
    assert c0["U2"] == c["U2"] and c0["X12"] == c["X12"] and c0["X34"] == c["X34"]
    ex.close()


def test_count_flops_mixed_split():
    s = ri.config(1)
    pk = ri.generate(s)
    ex = Exchange.from_system(s, precision="mixed")
    ex.set_CV(pk.C, pk.V)
    D = torch.from_numpy(pk.D).cuda()
    c = ex.count_flops(D)
    st = ex.stats()
    T, U2, Z = host_counts(s, pk, pk.D)
    assert c["T"] == T and c["U2"] == U2 and c["Z"] == Z
    assert 0 <= c["t_tc"] <= c["T"] and 0 <= c["z_tc"] <= c["Z"]
    assert 0 <= c["term1_tc"] <= c["X12"] - c["term2"]
    # the split follows the setup's choice of atoms: nothing counted where setup moved nothing
    for k, f in (("t_tc", "flops_t_tc"), ("z_tc", "flops_z_tc"), ("term1_tc", "flops_term1_tc")):
        assert (c[k] > 0) == (st[f] > 0), k
    ex.close()
