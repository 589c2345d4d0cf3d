// Counter-based Gaussian noise for the moving goals of the tracking task and
// for the exploration of the PPO policy.
//
// The 64-bit finaliser of SplitMix64 (Steele, Lea and Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014) hashes a key
// built from (seed, env, chain, step); two hashed words give four 24-bit
// uniforms u in (0, 1) and Box-Muller turns them into normal deviates.  No
// generator state is kept: any (env, chain, step) draws the same numbers
// whatever the launch configuration.
#pragma once

#include <cstdint>

namespace sg {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Three standard normal deviates for (seed, env, chain, step).
__device__ __forceinline__ void goal_noise(uint32_t seed, int env, int chain, int step,
                                           float& z0, float& z1, float& z2) {
  uint64_t key = mix64((uint64_t)seed + kGolden);
  key = mix64(key + kGolden + (uint64_t)(uint32_t)env);
  key = mix64(key + kGolden + (((uint64_t)(uint32_t)step << 2) | (uint64_t)chain));
  const uint64_t w0 = mix64(key + kGolden), w1 = mix64(key + 2 * kGolden);
  const float s = 1.f / 16777216.f;
  const float u0 = ((float)(w0 >> 40) + 0.5f) * s;
  const float u1 = ((float)((w0 >> 16) & 0xFFFFFFull) + 0.5f) * s;
  const float u2 = ((float)(w1 >> 40) + 0.5f) * s;
  const float u3 = ((float)((w1 >> 16) & 0xFFFFFFull) + 0.5f) * s;
  const float r0 = sqrtf(-2.f * logf(u0)), r1 = sqrtf(-2.f * logf(u2));
  float sn, cs;
  sincospif(2.f * u1, &sn, &cs);
  z0 = r0 * cs;
  z1 = r0 * sn;
  sincospif(2.f * u3, &sn, &cs);
  z2 = r1 * cs;
}

// Four standard normal deviates for (seed, env, block, step) of the policy's
// exploration noise (joint j: block j / 4, component j % 4).
__device__ __forceinline__ void action_noise(uint32_t seed, int env, int block, long long step,
                                             float (&z)[4]) {
  uint64_t key = mix64((uint64_t)seed + kGolden);
  key = mix64(key + kGolden + (uint64_t)(uint32_t)env);
  key = mix64(key + kGolden + (((uint64_t)step << 5) | (uint64_t)block));
  const uint64_t w0 = mix64(key + kGolden), w1 = mix64(key + 2 * kGolden);
  const float s = 1.f / 16777216.f;
  const float u0 = ((float)(w0 >> 40) + 0.5f) * s;
  const float u1 = ((float)((w0 >> 16) & 0xFFFFFFull) + 0.5f) * s;
  const float u2 = ((float)(w1 >> 40) + 0.5f) * s;
  const float u3 = ((float)((w1 >> 16) & 0xFFFFFFull) + 0.5f) * s;
  const float r0 = sqrtf(-2.f * logf(u0)), r1 = sqrtf(-2.f * logf(u2));
  float sn, cs;
  sincospif(2.f * u1, &sn, &cs);
  z[0] = r0 * cs;
  z[1] = r0 * sn;
  sincospif(2.f * u3, &sn, &cs);
  z[2] = r1 * cs;
  z[3] = r1 * sn;
}

}  // namespace sg
