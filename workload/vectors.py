"""Seeded start vectors.

The paper asks for a random start vector of norm 1 (Algorithm 1) without
naming a distribution.  Here it is uniform in [-1, 1), drawn from the
SplitMix64 generator (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used in counter mode:

    z   = (counter + 0x9E3779B97F4A7C15) mod 2^64
    z   = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9 mod 2^64
    z   = (z ^ (z >> 27)) * 0x94D049BB133111EB mod 2^64
    z   =  z ^ (z >> 31)
    x   = (z >> 11) * 2^-53                      in [0, 1)
    v[J] = 2x - 1                                (exact in binary64)

with counter = seed * 2^40 + J.  Every v[J] is exactly representable, so any
implementation of this recipe produces bit-identical vectors.  The vector is
returned unnormalised: the Lanczos routines normalise their start vector.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter):
    """SplitMix64 output for an array of uint64 counters (wrapping arithmetic)."""
    z = np.asarray(counter, dtype=np.uint64) + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def start_vector(n, seed=1234, start=0, dtype=np.float64):
    """Entries start .. start+n-1 of the seeded uniform[-1,1) start vector."""
    with np.errstate(over="ignore"):
        c = np.uint64(seed) * np.uint64(1 << 40) + np.uint64(start) + np.arange(n, dtype=np.uint64)
        z = splitmix64(c)
    x = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    v = 2.0 * x - 1.0
    return v.astype(dtype, copy=False)


def start_vector_into(out, seed=1234, chunk=1 << 25):
    """Fill a preallocated float64/float32 array with the seeded start vector, chunk by chunk."""
    n = out.shape[0]
    for s0 in range(0, n, chunk):
        m = min(chunk, n - s0)
        out[s0:s0 + m] = start_vector(m, seed=seed, start=s0, dtype=out.dtype)
    return out


def start_vector_at(indices, seed=1234):
    """Entries of the seeded start vector at arbitrary indices (float64)."""
    idx = np.asarray(indices, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = splitmix64(np.uint64(seed) * np.uint64(1 << 40) + idx)
    return 2.0 * ((z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)) - 1.0
