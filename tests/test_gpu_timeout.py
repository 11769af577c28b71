"""Bounded device waits: a wait that nothing completes gives up cleanly.

The sliced-GEMM kernel's waits are bounded by %globaltimer.  The test hook
rix_test_stalled_gemm runs it on a small problem whose MMA issuer waits on a
barrier that no thread or copy ever completes, with every wait limited to a
few milliseconds: the kernel must wait for its own bulk copies, free its
tensor memory and report RIX_ETIMEOUT, and the stream and context must stay
usable.  No fault, trap or hang is involved.
"""
import numpy as np
import pytest

import rix_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402


def _gemm_ok(st):
    g = torch.Generator().manual_seed(7)
    A = torch.randn(300, 200, generator=g, dtype=torch.float64)
    B = torch.randn(200, 170, generator=g, dtype=torch.float64)
    C = rix.gemm_sliced(A.cuda(), B.cuda(), 6, stream=st).cpu().numpy()
    scale = np.abs(A.numpy()).max(1)[:, None] * np.abs(B.numpy()).max(0)[None, :] * 200
    return (np.abs(C - (A @ B).numpy()) / scale).max()


def test_stalled_gemm_times_out_and_the_stream_stays_usable():
    st = torch.cuda.current_stream()
    for wait_ns in (2_000_000, 20_000_000):
        assert rix.stalled_gemm(wait_ns, stream=st) == rix.RIX_ETIMEOUT
    assert _gemm_ok(st) < 8 * 2.0 ** -42 + 2.0 ** -50


def test_wait_limit_out_of_range_is_rejected():
    assert rix.stalled_gemm(0) == rix.RIX_EINVAL
    assert rix.stalled_gemm(3_000_000_000) == rix.RIX_EINVAL


def test_context_reports_the_timeout_once():
    """A timed-out kernel of a context is reported by rix_check, then the context works again."""
    s = ri.config(0)
    pk = ri.generate(s)
    ex = rix.Exchange.from_system(s, precision="mixed")
    dev = torch.device("cuda")
    C, V, D = (torch.from_numpy(x).to(dev) for x in (pk.C, pk.V, pk.D))
    ex.set_CV(C, V)
    K0 = ex.build_K(D)
    ex.check()                                         # nothing pending
    assert rix.stalled_gemm(2_000_000, ctx=ex.ctx) == rix.RIX_OK
    with pytest.raises(rix.RixError) as e:
        ex.check()
    assert e.value.status == rix.RIX_ETIMEOUT
    ex.check()                                         # reported once, then cleared
    # a timeout left pending is reported by the next build instead
    assert rix.stalled_gemm(2_000_000, ctx=ex.ctx) == rix.RIX_OK
    torch.cuda.synchronize()
    with pytest.raises(rix.RixError) as e:
        ex.build_K(D)
    assert e.value.status == rix.RIX_ETIMEOUT
    K1 = ex.build_K(D)
    ex.check()
    assert torch.allclose(K0, K1, rtol=0, atol=1e-12 * K0.abs().max().item())
    ex.close()
