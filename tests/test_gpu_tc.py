"""Sliced BF16 tensor-core GEMM (rix_gemm_sliced) against exact and FP64 references.

* Integer operands of two digits (14 bits) with n_slices = 3 keep every
  digit pair, and every pair lands in one of the exactly accumulated
  diagonals, so the product is exact: a bit-exact check of the tensor-core
  accumulation, the operand layouts and the fixed-point fold.
* Random FP64 operands: error within a small multiple of 2^(-7 S) of
  (row scale x column scale x K), plus 2^-50 of it for the FP32 accumulation
  of the terms 2^-35 and more below the leading one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2403_10343_gb300 import rix  # noqa: E402


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (200, 100, 300), (129, 65, 33), (300, 200, 784), (130, 300, 1700)])
def test_exact_integers(M, N, K):
    r = np.random.default_rng(M * 7 + N + K)
    A = r.integers(-(1 << 13), 1 << 13, size=(M, K)).astype(np.int64)
    B = r.integers(-(1 << 13), 1 << 13, size=(K, N)).astype(np.int64)
    ref = A @ B                                   # exact in int64 (< 2^53)
    At = torch.from_numpy(A.astype(np.float64)).cuda()
    Bt = torch.from_numpy(B.astype(np.float64)).cuda()
    C = rix.gemm_sliced(At, Bt, 3).cpu().numpy()  # 14-bit integers: 2 digits, all pairs kept
    assert np.array_equal(C, ref.astype(np.float64))


@pytest.mark.parametrize("S", [3, 4, 6, 7])
def test_random_fp64_accuracy(S):
    r = np.random.default_rng(S)
    M, N, K = 257, 190, 500
    A = r.normal(size=(M, K)) * np.exp(r.normal(size=(M, 1)))
    B = r.normal(size=(K, N)) * np.exp(r.normal(size=(1, N)))
    ref = A @ B
    C = rix.gemm_sliced(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), S).cpu().numpy()
    scale = np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :] * K
    err = np.abs(C - ref) / scale
    print(f"S={S}: max error {err.max():.3e} = 2^{np.log2(err.max()):.1f}")
    assert err.max() < 8 * 2.0 ** (-7 * S) + 2.0 ** (-50), err.max()
