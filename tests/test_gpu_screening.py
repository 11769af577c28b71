"""Product screening (rix_options.product_tau) on the (H2O)64 cluster.

The paper screens products of blocks by their norms (Sec. "Evaluation of the
EXX matrix in real space").  With product_tau = 0 the build is unchanged
(bitwise, FP64 path).  With product_tau > 0 the T and Z stages skip the
block products whose max-norms multiply to less than it: the counted FLOPs
drop, and K moves away from the oracle's unscreened K by an amount that is
measured here (and must stay small against the threshold).
"""
import numpy as np
import pytest

import rix_inputs as ri
from oracle.oracle import Oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402
from workloads import rel, rows_of  # noqa: E402

ROWS = [0, 1, 2, 93, 94, 95]


def _run(s, pk, prec, ptau):
    ex = rix.Exchange.from_system(s, precision=prec, product_tau=ptau)
    dev = torch.device("cuda")
    ex.set_CV(torch.from_numpy(pk.C).to(dev), torch.from_numpy(pk.V).to(dev))
    D = torch.from_numpy(pk.D).to(dev)
    K = ex.build_K(D)
    E = ex.energy(D, K).item()
    fl = ex.count_flops(D)
    keys = ex.k_keys()
    out = K.cpu().numpy(), E, fl["T"] + fl["Z"], keys
    ex.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_product_screening(prec):
    s = ri.config(1)
    pk = ri.generate(s)
    K0, E0, f0, keys = _run(s, pk, prec, 0.0)
    if prec == "fp64":
        K00, E00, _, _ = _run(s, pk, prec, 0.0)
        base = rix.Exchange.from_system(s)
        assert np.array_equal(K0, K00)
        base.close()
    o = Oracle(s)
    o.set_data(pk.C, pk.V, pk.D)
    kr = o.kpattern(ROWS)
    Kr = o.build_K()
    for ptau in (1e-10, 1e-8):
        K, E, f, _ = _run(s, pk, prec, ptau)
        sub_keys, sub = rows_of(s, keys, K, ROWS)
        assert np.array_equal(sub_keys, kr)
        err = rel(sub, Kr)
        print(f"{prec} product_tau {ptau:g}: T+Z FLOPs {f:.3e} of {f0:.3e}, K rows vs unscreened oracle "
              f"{err:.2e}, E_x change {E - E0:.2e} Ha")
        assert f < f0
        assert err < 1e4 * ptau + (1e-8 if prec == "mixed" else 1e-12)
