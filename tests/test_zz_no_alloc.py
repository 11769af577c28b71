"""rix_energy_noalloc against rix_energy, through the C ABI, two calls in a row.

The no-allocation variant exists for callers that cannot allocate device
memory when they need the energy (their caching allocator holds the free
memory, or their loop forbids allocation).  It must give the same energy as
the regular entry point, including on a second call that reuses the shared
fixed scratch array left over from the first.
"""
import numpy as np
import pytest

import rix_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402

E_TOL = 1e-12


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("cfg", [0, 1])
def test_energy_noalloc_matches_energy(cfg):
    s = ri.config(cfg)
    pk = ri.generate(s)
    ex = rix.Exchange.from_system(s)
    C, V, D = _dev(pk.C), _dev(pk.V), _dev(pk.D)
    ex.set_CV(C, V)
    K = ex.build_K(D)
    ref = torch.empty(1, dtype=torch.float64, device="cuda")
    got = torch.empty(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        # second call: a different D, so stale scratch from the first would show
        Dc = D if call == 0 else 0.5 * D
        Kc = K if call == 0 else ex.build_K(Dc)
        rix.energy(ex.ctx, Dc, Kc, ref)
        got.fill_(float("nan"))
        rix.energy_noalloc(ex.ctx, Dc, Kc, got)
        torch.cuda.synchronize()
        e_ref, e_got = ref.item(), got.item()
        assert np.isfinite(e_got)
        assert abs(e_got - e_ref) <= E_TOL * abs(e_ref), (call, e_got, e_ref)
    ex.close()
