// rng.cuh -- counter-based random rotation angles for the noise maps (Sec. 1).
#pragma once

#include "common.cuh"

namespace fm {

// SplitMix64 at a counter (Steele, Lea & Flood 2014): state `seed` advanced
// (index + 1) times by the golden gamma, then the 64-bit finaliser.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void rot_sincos(float two_u, float *s, float *c) { sincospif(two_u, s, c); }
__device__ __forceinline__ void rot_sincos(double two_u, double *s, double *c) { sincospi(two_u, s, c); }


// Rotation of pixel (y, x) of realisation r: gamma * exp(2 i alpha),
// alpha = pi u, u = top 24 bits of SplitMix64 at (r n + y) n + x, times 2^-24.
template <typename T>
__device__ __forceinline__ void rotate_shear(T &a, T &c, uint64_t seed, long r, int y, int x, int n)
{
    const uint64_t ctr = ((uint64_t)r * (uint64_t)n + (uint64_t)y) * (uint64_t)n + (uint64_t)x;
    const T u = (T)(splitmix64_at(seed, ctr) >> 40) * (T)(1.0 / 16777216.0);
    T sn, cs;
    rot_sincos((T)2 * u, &sn, &cs);
    const T ra = a * cs - c * sn;
    const T rc = a * sn + c * cs;
    a = ra;
    c = rc;
}

}  // namespace fm
