"""RI-LVL coefficient fit on the GPU (rix_fit_C) against the oracle (oracle/rifit.py).

* Even-tempered aux basis (a well-conditioned pair metric), integrals
  (ij|nu) = V^{IJ} C0: the device fit returns C0 and the oracle's fit, to the
  metric's condition number times rounding; the result is exactly
  pair-symmetric, so rix_set_CV accepts it, and the exchange build from the
  fitted C equals the build from C0 to the FP64 bar.
* The workload's own aux basis (numerically singular metrics) with a Tikhonov
  shift lambda: the device fit matches the oracle's fit with the same shift.
"""
import numpy as np
import pytest

import rix_inputs as ri
from oracle.rifit import fit_C, metric

from rifit_systems import eri_from, even_tempered_waters

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("periodic", [False, True])
def test_fit_recovers_C_and_matches_oracle(periodic):
    o = [[0.0, 0.0, 0.0], [2.9, 0.4, -0.3]] if not periodic else [[1.0, 1.2, 0.8], [3.9, 3.1, 3.3]]
    s = even_tempered_waters(o, 23, cell_side=6.0 if periodic else None, cutoff_ang=4.5 if periodic else None)
    pk = ri.generate(s)
    cond = max(np.linalg.cond(metric(s, pk, p)) for p in range(pk.n_pairs))
    eri = eri_from(s, pk, pk.C)
    ex = rix.Exchange.from_system(s)
    V = _dev(pk.V)
    C = rix.fit_C(ex.ctx, V, _dev(eri))
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    ref = fit_C(s, pk, eri)
    scale = np.abs(pk.C).max()
    tol = 100 * cond * 2.0 ** -52
    print(f"periodic={periodic}: max cond {cond:.2e}, vs C0 {np.abs(got - pk.C).max() / scale:.2e}, "
          f"vs oracle {np.abs(got - ref).max() / scale:.2e}")
    assert np.abs(got - pk.C).max() < tol * scale
    assert np.abs(got - ref).max() < tol * scale
    ex.set_CV(C, V)                                     # exactly pair-symmetric, or RIX_ENOTSYM
    D = _dev(pk.D)
    K1 = ex.build_K(D).cpu().numpy()
    ex.set_CV(_dev(pk.C), V)
    K0 = ex.build_K(D).cpu().numpy()
    assert np.linalg.norm(K1 - K0) / np.linalg.norm(K0) < tol
    ex.close()


def test_tikhonov_fit_on_the_workload_basis():
    s = ri.config(0)
    pk = ri.generate(s)
    lam = 1e-6
    rng = np.random.default_rng(5)
    eri = eri_from(s, pk, pk.C)
    ex = rix.Exchange.from_system(s)
    got = rix.fit_C(ex.ctx, _dev(pk.V), _dev(eri), lam).cpu().numpy()
    ref = fit_C(s, pk, eri, lam)
    # both solve the same shifted system; their difference is bounded by its condition number
    cond = max(np.linalg.cond(metric(s, pk, p, lam)) for p in rng.choice(pk.n_pairs, 20, replace=False))
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"Tikhonov lambda {lam}: cond ~{cond:.1e}, device vs oracle {err:.2e}")
    assert err < 100 * cond * 2.0 ** -52
    ex.close()
