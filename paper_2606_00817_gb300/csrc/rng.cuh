// rng.cuh -- counter-based uniforms from SplitMix64 (Steele, Lea and Flood's
// 64-bit mixing function): draw m of (seed, a, b) is mix(key(seed, a, b) + m),
// so any draw can be regenerated on its own, on any thread.
#pragma once
#include <cstdint>

namespace ddf {

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t rng_key(uint64_t seed, uint64_t a, uint64_t b) {
  return sm64(sm64(seed ^ 0x5DEECE66Dull) + a) ^ (b * 0x2545F4914F6CDD1Dull);
}

// Uniform in [0, 1) from the top 24 bits (exact in float32).
__device__ __forceinline__ float rng_u01(uint64_t key, int m) {
  return static_cast<float>(sm64(key + static_cast<uint64_t>(m)) >> 40) * (1.0f / 16777216.0f);
}

}  // namespace ddf
