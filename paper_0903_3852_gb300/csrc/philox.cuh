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

// Each round's two 32 x 32 -> 64-bit products are written as 64-bit
// multiplies, one wide multiply-add instruction each.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;
    const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y,
                   (uint32_t)p0);
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
    const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;
    const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k[2 * round], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ K.k[2 * round + 1], (uint32_t)p0);
  }
  return c;
}

__device__ __forceinline__ uint2 seed_to_key(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ float uniform24(uint32_t w) {
  return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f;  // 2^-24
}

// sqrt(L) for the Box-Muller radius by the hardware square-root
// approximation (one instruction; L = 0, reached when u0 = 1, gives 0).
__device__ __forceinline__ float radius(float L) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(L));
  return r;
}

__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float &z0, float &z1) {
  const float u0 = uniform24(w0);
  const float rho = radius(-2.0f * logf(u0));
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

// Box-Muller of the Josephson kernels, two shortcuts against box_muller:
//  * the angle's sine and cosine from a table: the angle 2 pi u1,
//    u1 = (j + 1) 2^-24 with j = w1 >> 8, is split into the table angle
//    2 pi q / 1024 (q = the top 10 bits of j) and a remainder
//    b = 2 pi ((j mod 2^14) + 1) 2^-24 in (0, 2 pi / 1024]; sin b = b and
//    cos b = 1 - b^2/2 (the next terms are below 4e-8), and the
//    angle-addition formulas combine them with the table entry (within
//    about 1e-7 of the exact values);
//  * ln u0 from the hardware base-2 logarithm (lg2.approx, one instruction)
//    times ln 2.  Its error is absolute, so the radius sqrt(-2 ln u0) keeps
//    a relative accuracy of ~1e-7 for u0 well below 1 and loses it as
//    u0 -> 1 (radius -> 0); the radius error stays below ~5e-4 everywhere
//    (the bound the tests check on all 2^24 values of u0).  A slightly
//    positive log of a u0 just below 1 is clamped to a zero radius.
// tab[q] = cos(2 pi q / 1024) and tab[kBmTable + q] = sin(2 pi q / 1024),
// q = 0 .. 1023, filled by fill_bm_table (shared memory of the calling
// kernel, 8 KB); separate cos and sin arrays, so that two lookups can land in
// the two halves of a packed FP32 pair.
constexpr int kBmTable = 1024;

__device__ __forceinline__ void fill_bm_table(float *tab) {
  for (int q = threadIdx.x; q < kBmTable; q += blockDim.x) {
    float sn, cs;
    sincospif((float)q * 0.001953125f, &sn, &cs);  // q / 512
    tab[q] = cs;
    tab[kBmTable + q] = sn;
  }
}

__device__ __forceinline__ void box_muller_tab(uint32_t w0, uint32_t w1, const float *tab, float &z0,
                                               float &z1) {
  const float u0 = fmaf((float)(w0 >> 8), 5.9604644775390625e-8f, 5.9604644775390625e-8f);  // exact
  float l2;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(u0));
  const float rho = radius(fmaxf(-1.38629436111989061883f * l2, 0.0f));  // -2 ln 2 log2(u0)
  const float2 t = make_float2(tab[w1 >> 22], tab[kBmTable + (w1 >> 22)]);
  const float b = fmaf((float)((w1 >> 8) & 0x3FFFu), 3.7450702829239308e-7f, 3.7450702829239308e-7f);  // 2 pi 2^-24
  const float cb = fmaf(-0.5f * b, b, 1.0f);
  z0 = rho * fmaf(t.x, cb, -t.y * b);
  z1 = rho * fmaf(t.y, cb, t.x * b);
}

// box_muller_tab for two word pairs at once (the same words of two paths) on
// packed FP32 pairs: Z0 = (z0 of A, z0 of B), Z1 = (z1 of A, z1 of B), the
// same roundings as box_muller_tab element by element.
__device__ __forceinline__ void box_muller_tab2(uint32_t a0, uint32_t a1, uint32_t b0, uint32_t b1,
                                                const float *tab, float2 &Z0, float2 &Z1) {
  const float2 q = make_float2(5.9604644775390625e-8f, 5.9604644775390625e-8f);  // 2^-24
  const float2 u0 = __ffma2_rn(make_float2((float)(a0 >> 8), (float)(b0 >> 8)), q, q);
  float la, lb;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(la) : "f"(u0.x));
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lb) : "f"(u0.y));
  const float2 L = __fmul2_rn(make_float2(-1.38629436111989061883f, -1.38629436111989061883f),
                              make_float2(la, lb));
  const float2 rho = make_float2(radius(fmaxf(L.x, 0.0f)), radius(fmaxf(L.y, 0.0f)));
  const float2 c = make_float2(3.7450702829239308e-7f, 3.7450702829239308e-7f);  // 2 pi 2^-24
  const float2 b =
      __ffma2_rn(make_float2((float)((a1 >> 8) & 0x3FFFu), (float)((b1 >> 8) & 0x3FFFu)), c, c);
  const float2 cb = __ffma2_rn(__fmul2_rn(make_float2(-0.5f, -0.5f), b), b, make_float2(1.0f, 1.0f));
  const float2 tx = make_float2(tab[a1 >> 22], tab[b1 >> 22]);
  const float2 ty = make_float2(tab[kBmTable + (a1 >> 22)], tab[kBmTable + (b1 >> 22)]);
  const float2 nb = make_float2(-b.x, -b.y);
  Z0 = __fmul2_rn(rho, __ffma2_rn(tx, cb, __fmul2_rn(ty, nb)));
  Z1 = __fmul2_rn(rho, __ffma2_rn(ty, cb, __fmul2_rn(tx, b)));
}

// Element k (0..3) of a 4-vector without dynamic register indexing.
__device__ __forceinline__ float pick4(const float (&z)[4], int k) {
  return k == 0 ? z[0] : (k == 1 ? z[1] : (k == 2 ? z[2] : z[3]));
}

}  // namespace sde
