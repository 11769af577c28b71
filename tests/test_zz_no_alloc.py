"""rix_energy_noalloc against rix_energy, through the C ABI, two calls in a row.

Some callers cannot allocate device memory at the point where they need the
energy: a framework whose caching allocator already holds the GPU's free
memory, or an SCF loop that forbids allocation (and the synchronisation it can
cause).  rix_energy_noalloc serves them with a fixed library-owned scratch
array.  It must give exactly the energy of the regular entry point (the same
kernels in the same reduction order), also when a call with fewer partial sums
follows one with more (stale partial sums left in the shared array must not
leak in), and it must not change the device memory in use.
"""
import numpy as np
import pytest

import rix_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _energies(ex, D, K):
    ref = torch.empty(1, dtype=torch.float64, device="cuda")
    got = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    rix.energy(ex.ctx, D, K, ref)
    torch.cuda.synchronize()
    used, free = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
    rix.energy_noalloc(ex.ctx, D, K, got)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == used
    assert torch.cuda.mem_get_info()[0] == free
    return ref.item(), got.item()


def test_energy_noalloc_matches_energy_larger_then_smaller():
    # the 192-atom cluster fills more of the shared array than the 24-atom one that follows
    for cfg, scale in ((1, 1.0), (0, 0.5)):
        s = ri.config(cfg)
        pk = ri.generate(s)
        ex = rix.Exchange.from_system(s)
        C, V, D = _dev(pk.C), _dev(pk.V), scale * _dev(pk.D)
        ex.set_CV(C, V)
        K = ex.build_K(D)
        for call in range(2):
            Dc = D if call == 0 else 0.75 * D
            Kc = K if call == 0 else ex.build_K(Dc)
            e_ref, e_got = _energies(ex, Dc, Kc)
            assert np.isfinite(e_got)
            assert e_got == e_ref, (cfg, call, e_got, e_ref)
        ex.close()
