"""Counter-based random numbers (SplitMix64) for seeded synthetic inputs.

SplitMix64 is the 64-bit mixing function of Steele, Lea and Flood,
"Fast splittable pseudorandom number generators" (OOPSLA 2014), in the form
popularised by Vigna: add the golden-ratio increment 0x9E3779B97F4A7C15, then
two xor-shift-multiply rounds (shifts 30, 27, multipliers 0xBF58476D1CE4E5B9,
0x94D049BB133111EB) and a final xor-shift by 31.  All arithmetic is modulo
2**64.

A stream of numbers is addressed by (seed, stream, i):

    key            = splitmix64(splitmix64(seed) + stream)
    counter_u64(i) = splitmix64(key + i)

The CUDA library implements the same definition independently for the random
test vectors it draws at set-up time (``uniform_pm1`` of stream
``STREAM_TESTVEC``), so both sides produce bit-identical values.
"""

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers: one per kind of drawn quantity.
STREAM_GAUGE = 1
STREAM_SPINOR = 2
STREAM_TESTVEC = 3
STREAM_GAUGE_TRANSFORM = 4
STREAM_Z2 = 5


def splitmix64(x):
    """SplitMix64 mix of a uint64 array (or scalar), modulo 2**64."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed, stream):
    """Key of stream ``stream`` under ``seed``."""
    with np.errstate(over="ignore"):
        return splitmix64(splitmix64(np.uint64(seed)) + np.uint64(stream))


def counter_u64(seed, stream, i):
    """The i-th uint64 of (seed, stream); ``i`` may be an array of indices."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        return splitmix64(key + np.asarray(i, dtype=np.uint64))


def uniform_pm1(u):
    """Map uint64 -> k * 2**-52 - 1 with k = u >> 11, a value in [-1, 1).

    Every value is exactly representable in binary64, so any implementation
    of the same integer steps gives bit-identical results.
    """
    k = (np.asarray(u, dtype=np.uint64) >> np.uint64(11)).astype(np.float64)
    return k * (2.0 ** -52) - 1.0


def uniform_open01(u):
    """Map uint64 -> (k + 1) * 2**-53 with k = u >> 11, a value in (0, 1]."""
    k = (np.asarray(u, dtype=np.uint64) >> np.uint64(11)).astype(np.float64)
    return (k + 1.0) * (2.0 ** -53)


def gaussian(seed, stream, j):
    """Standard normal deviates by Box-Muller from counters 2j and 2j+1."""
    j = np.asarray(j, dtype=np.uint64)
    u1 = uniform_open01(counter_u64(seed, stream, j * np.uint64(2)))
    u2 = uniform_open01(counter_u64(seed, stream, j * np.uint64(2) + np.uint64(1)))
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
