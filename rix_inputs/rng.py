"""Counter-based random numbers for the synthetic inputs.

Every random value used by the input generators is a pure function of
(seed, stream, counter), so any element of any packed array can be
regenerated on its own (the oracle's row-subset mode regenerates only the
blocks it needs).

Hash: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), applied to
``seed * K1 + stream * K2 + counter``.  Normal deviates use the Box-Muller
transform on two 53-bit uniforms drawn from counters 2c and 2c+1.
"""
import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_K_SEED = np.uint64(0xD1B54A32D192ED03)
_K_STREAM = np.uint64(0x8CB92BA72F3D8DD7)


def splitmix64(x):
    """SplitMix64 finaliser of (x + golden gamma); uint64 array in, uint64 out."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GOLDEN).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _base(seed, stream):
    with np.errstate(over="ignore"):
        return np.uint64(seed) * _K_SEED + np.uint64(stream) * _K_STREAM


def uniform(seed, stream, counters):
    """Uniform doubles in [0, 1) with 53 random bits, one per counter."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = splitmix64(_base(seed, stream) + c)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed, stream, counters):
    """Standard normal deviates (Box-Muller), one per counter."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        c2 = c * np.uint64(2)
        u1 = uniform(seed, stream, c2)
        u2 = uniform(seed, stream, c2 + np.uint64(1))
    u1 = 1.0 - u1  # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# Stream identifiers (fixed; documented in the design notes).
STREAM_C = 1
STREAM_D = 2
STREAM_AUX = 3
STREAM_GEOM = 4
