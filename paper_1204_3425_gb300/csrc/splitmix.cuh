// Seeded uniform [-1, 1) start-vector elements: SplitMix64 (Steele, Lea,
// Flood 2014) in counter mode, counter = seed * 2^40 + i; the top 53 bits of
// the output give x in [0, 1), v = 2x - 1 (exact in binary64).  Used by the
// fill kernel and by the queued solver, which draws each task's start vector
// in place, so both give the same vector for the same seed.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hub {

__device__ __forceinline__ double splitmix_uniform(unsigned long long seed, long long i) {
    unsigned long long z = seed * (1ull << 40) + (unsigned long long)i + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double x = (double)(z >> 11) * 0x1p-53;
    return 2.0 * x - 1.0;
}

}  // namespace hub
