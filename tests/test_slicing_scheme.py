"""The arithmetic of the error-free slicing behind the tensor-core GEMM, on the CPU.

The GPU kernel's correctness rests on three facts that need no GPU to check:

* balanced base-2^7 digits: every value x of a row with |x| < 2^e is written
  as sign(x) * sum_t d_t 2^(-7(t+1)) * 2^e with d_0 in [0, 128] and the other
  digits in [-64, 63], and the remainder is at most half a unit of the last
  digit;
* the integer bounds: a slice product is at most 128*128 on the leading
  diagonal, 128*64 with one leading digit and 64*64 otherwise, so each of the
  five exactly accumulated diagonals stays below 2^24 over 512 K values (the
  FP32 accumulators of the tensor cores are then exact);
* the result: the sum over diagonals s + t <= S + 1 of the slice products,
  rescaled, is A B within about 2^(-7S) of (row scale x column scale x K).

Here the digits are formed with Python integers from the same definition
(scale by the row's power of two, cut the 64-bit fraction, round the last
digit, fold digits >= 64 downwards with a carry) and the products are exact
integers, so the checks are exact.
"""
import math
import struct

import numpy as np
import pytest

KC, GROUP = 32, 16  # the kernel's K stage and stages per accumulation group (512 K values)


def row_exponent(row):
    m = max((abs(float(x)) for x in row), default=0.0)
    return math.frexp(m)[1] if m > 0 else -2000  # |x| < 2^e


def fraction64(x, e):
    """|x| / 2^e as a 64-bit fixed-point integer (exact for the doubles used here)."""
    b = struct.unpack("<Q", struct.pack("<d", abs(x)))[0]
    ex = (b >> 52) & 0x7FF
    if ex == 0:
        return 0
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = 12 + (ex - 1023) - e
    return (m << sh) & ((1 << 64) - 1) if sh >= 0 else (m >> -sh if sh > -64 else 0)


def balanced_digits(x, e, S):
    fr = fraction64(x, e)
    carry = (fr >> (63 - 7 * S)) & 1
    d = [0] * S
    for t in range(S - 1, 0, -1):
        c = ((fr >> (57 - 7 * t)) & 127) + carry
        carry = 1 if c >= 64 else 0
        d[t] = c - (carry << 7)
    d[0] = (fr >> 57) + carry
    sg = -1 if x < 0 else 1
    return [sg * v for v in d]


@pytest.mark.parametrize("S", [3, 5, 6, 7])
def test_balanced_digits_ranges_and_remainder(S):
    rng = np.random.default_rng(S)
    for _ in range(3000):
        x = float(rng.standard_normal() * 2.0 ** rng.integers(-40, 40))
        e = math.frexp(abs(x))[1] + int(rng.integers(0, 3))
        d = balanced_digits(x, e, S)
        assert 0 <= abs(d[0]) <= 128 and all(-64 <= v * (1 if x >= 0 else -1) <= 63 for v in d[1:])
        # value represented, in units of the last digit, against the exact fraction
        got = sum(v * 128 ** (S - 1 - t) for t, v in enumerate(d))
        exact = (1 if x >= 0 else -1) * fraction64(x, e) / 2.0 ** (64 - 7 * S)
        assert abs(got - exact) <= 0.5 + 1e-9


def diag_bound(a):
    """Largest |sum over one K value| of diagonal a (pairs (s, a - s))."""
    if a == 0:
        return 128 * 128
    return 2 * 128 * 64 + (a - 1) * 64 * 64


def test_exact_accumulation_bounds():
    for a in range(5):
        assert diag_bound(a) * GROUP * KC < 2 ** 24
    # the bound is attained: digits at their extremes on every K value
    lead, rest = 128, -64
    d = [lead] + [rest] * 6
    for a in range(1, 5):
        worst = sum(abs(d[s] * d[a - s]) for s in range(a + 1))
        assert worst == diag_bound(a)


@pytest.mark.parametrize("S", [3, 4, 5, 6])
def test_sliced_product_error(S):
    rng = np.random.default_rng(10 + S)
    M, N, K = 7, 5, 40
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-8, 8, (M, K)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-8, 8, (K, N)))
    eA = [row_exponent(A[i]) for i in range(M)]
    eB = [row_exponent(B[:, j]) for j in range(N)]
    dA = [[balanced_digits(A[i, k], eA[i], S) for k in range(K)] for i in range(M)]
    dB = [[balanced_digits(B[k, j], eB[j], S) for k in range(K)] for j in range(N)]
    worst = 0.0
    for i in range(M):
        for j in range(N):
            # exact integer sum of the kept slice products, diagonal by diagonal
            tot = 0
            for a in range(S):  # the kept diagonals: s + t = a <= S - 1 (0-based digits)
                diag = sum(dA[i][k][s] * dB[j][k][a - s] for k in range(K) for s in range(a + 1))
                assert a >= 5 or abs(diag) <= diag_bound(a) * K
                tot += diag * 128 ** (2 * S - 2 - a)
            c = tot * 2.0 ** (eA[i] + eB[j] - 7 * (2 * S))
            exact = float(np.dot(A[i].astype(np.longdouble), B[:, j].astype(np.longdouble)))
            scale = 2.0 ** (eA[i] + eB[j]) * K
            worst = max(worst, abs(c - exact) / scale)
    print(f"S={S}: max error {worst:.3e} = 2^{math.log2(worst):.1f} of row x column x K")
    assert worst < 2.0 ** (-7 * S)
