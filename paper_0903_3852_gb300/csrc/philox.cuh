// philox.cuh -- counter-based Gaussian noise on the device.
//
// Philox4x32-10 from Salmon, Moraes, Dror & Shaw, "Parallel random numbers:
// as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplies with
// the multipliers 0xD2511F53 and 0xCD9E8D57, the round permutation
// (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), and the key bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85 after every round.  It replaces the
// per-thread xorshift generator of Sec. 4.1: the noise of step n is a pure
// function of (step, path, point) so that runs split at any step reproduce
// the unsplit run bit for bit.
//
// Uniforms take the top 24 bits of a word: u = ((w >> 8) + 1) * 2^-24, in
// (0, 1] and exact in FP32.  Box-Muller (Sec. 4.1, two uniforms -> two
// Gaussians): z0 = sqrt(-2 ln u0) cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1).
// The angle u1 is a 24-bit fraction of a turn, so its sine and cosine are
// taken from the fixed-point value ((w1 >> 8) + 1) * 2^8 directly.
#pragma once

#include <stdint.h>

#include "turns.cuh"

namespace sde {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of a seed (k + r W for round r), computed once on the
// host and passed to kernels as parameters, so that the rounds read them as
// constant operands.
struct PhiloxKeys {
  uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_round_keys(uint64_t seed) {
  PhiloxKeys K;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0;
    K.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &K) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ K.k[2 * round], lo1, hi0 ^ c.w ^ K.k[2 * round + 1], lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_to_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float uniform24(uint32_t w) {
  return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f;  // 2^-24
}

__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float &z0, float &z1) {
  const float u0 = uniform24(w0);
  // sqrt(L) as L rsqrt(L) (two instructions, within 2 ulp); L = 0 exactly
  // when u0 = 1, which 1 in 2^24 draws hit
  const float L = -2.0f * logf(u0);
  const float rho = L > 0.0f ? L * rsqrtf(L) : 0.0f;
  float s, c;
  sincos_turns(((w1 >> 8) + 1u) << 8, s, c);
  z0 = rho * c;
  z1 = rho * s;
}

// Four Gaussians of one Philox block: steps 4g..4g+3 of a stream.
__device__ __forceinline__ void gauss4(uint32_t g, uint32_t c1, uint32_t c2, uint32_t tag,
                                       uint2 key, float (&z)[4]) {
  const uint4 r = philox4x32_10(make_uint4(g, c1, c2, tag), key);
  box_muller(r.x, r.y, z[0], z[1]);
  box_muller(r.z, r.w, z[2], z[3]);
}

// gauss4 with precomputed round keys.
__device__ __forceinline__ void gauss4(uint32_t g, uint32_t c1, uint32_t c2, uint32_t tag,
                                       const PhiloxKeys &K, float (&z)[4]) {
  const uint4 r = philox4x32_10(make_uint4(g, c1, c2, tag), K);
  box_muller(r.x, r.y, z[0], z[1]);
  box_muller(r.z, r.w, z[2], z[3]);
}

// The one Gaussian of step n of a stream, identical to element n & 3 of
// gauss4 for the block n / 4 (only the Box-Muller pair that holds it is
// evaluated).
__device__ __forceinline__ float gauss1(int64_t n, uint32_t c1, uint32_t c2, uint32_t tag, uint2 key) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(n >> 2), c1, c2, tag), key);
  const bool hi = (n & 2) != 0;
  float z0, z1;
  box_muller(hi ? r.z : r.x, hi ? r.w : r.y, z0, z1);
  return (n & 1) ? z1 : z0;
}

// gauss1 with precomputed round keys.
__device__ __forceinline__ float gauss1(int64_t n, uint32_t c1, uint32_t c2, uint32_t tag,
                                        const PhiloxKeys &K) {
  const uint4 r = philox4x32_10(make_uint4((uint32_t)(n >> 2), c1, c2, tag), K);
  const bool hi = (n & 2) != 0;
  float z0, z1;
  box_muller(hi ? r.z : r.x, hi ? r.w : r.y, z0, z1);
  return (n & 1) ? z1 : z0;
}

// Element k (0..3) of a 4-vector without dynamic register indexing.
__device__ __forceinline__ float pick4(const float (&z)[4], int k) {
  return k == 0 ? z[0] : (k == 1 ? z[1] : (k == 2 ? z[2] : z[3]));
}

}  // namespace sde
