// turns.cuh -- sin and cos of a phase held as 32-bit fixed-point turns
// (2^32 units per 2 pi), the representation of the Kuramoto kernels.
//
// The top two bits (rounded) pick the nearest quarter turn q; the remainder
// r is an exact int32 in [-2^29, 2^29), i.e. x = 2 pi r / 2^32 in [-pi/4,
// pi/4).  sin x and cos x come from minimax polynomials on that interval,
// fitted for this library by linear programming on a dense grid (odd degree
// 7 for sin, even degree 8 for cos; FP32 Horner evaluation within 7e-8 of
// the exact values), and the quarter turn is applied by swapping and
// negating: sin(q pi/2 + x) = (sin x, cos x, -sin x, -cos x)[q], cos(q pi/2 +
// x) = (cos x, -sin x, -cos x, sin x)[q].  No range reduction of a float
// is needed, so the cost and the error do not depend on the phase.
#pragma once

#include <stdint.h>

namespace sde {

__device__ __forceinline__ void sincos_turns(uint32_t th, float &sn, float &cs) {
  const uint32_t q = (th + 0x20000000u) >> 30;
  const float x = (float)(int32_t)(th - (q << 30)) * 1.46291807926715968e-9f;  // 2 pi / 2^32
  const float x2 = x * x;
  const float s = fmaf(x * x2, fmaf(x2, fmaf(x2, -1.956071210e-4f, 8.332642727e-3f), -1.666666716e-1f), x);
  const float c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 2.456674520e-5f, -1.388842822e-3f), 4.166666791e-2f),
                                -0.5f),
                       1.0f);
  const float ss = (q & 1u) ? c : s;
  const float cc = (q & 1u) ? s : c;
  sn = (q & 2u) ? -ss : ss;
  cs = ((q + 1u) & 2u) ? -cc : cc;
}

// sincos_turns of two phases at once, the polynomials on packed FP32 pairs
// (the same roundings as sincos_turns element by element).
__device__ __forceinline__ void sincos_turns2(uint32_t ta, uint32_t tb, float2 &sn, float2 &cs) {
  const uint32_t qa = (ta + 0x20000000u) >> 30, qb = (tb + 0x20000000u) >> 30;
  const float2 x = __fmul2_rn(make_float2((float)(int32_t)(ta - (qa << 30)), (float)(int32_t)(tb - (qb << 30))),
                              make_float2(1.46291807926715968e-9f, 1.46291807926715968e-9f));
  const float2 x2 = __fmul2_rn(x, x);
  const float2 ps = __ffma2_rn(__ffma2_rn(x2, make_float2(-1.956071210e-4f, -1.956071210e-4f),
                                          make_float2(8.332642727e-3f, 8.332642727e-3f)),
                               x2, make_float2(-1.666666716e-1f, -1.666666716e-1f));
  const float2 s = __ffma2_rn(__fmul2_rn(x, x2), ps, x);
  float2 pc = __ffma2_rn(x2, make_float2(2.456674520e-5f, 2.456674520e-5f),
                         make_float2(-1.388842822e-3f, -1.388842822e-3f));
  pc = __ffma2_rn(x2, pc, make_float2(4.166666791e-2f, 4.166666791e-2f));
  pc = __ffma2_rn(x2, pc, make_float2(-0.5f, -0.5f));
  const float2 c = __ffma2_rn(x2, pc, make_float2(1.0f, 1.0f));
  const float ssa = (qa & 1u) ? c.x : s.x, cca = (qa & 1u) ? s.x : c.x;
  const float ssb = (qb & 1u) ? c.y : s.y, ccb = (qb & 1u) ? s.y : c.y;
  sn = make_float2((qa & 2u) ? -ssa : ssa, (qb & 2u) ? -ssb : ssb);
  cs = make_float2(((qa + 1u) & 2u) ? -cca : cca, ((qb + 1u) & 2u) ? -ccb : ccb);
}

// sincos_turns of n phases, two at a time on packed pairs (one alone if n is
// odd).
template <int N>
__device__ __forceinline__ void sincos_turns_n(const uint32_t (&th)[N], float (&sn)[N], float (&cs)[N]) {
#pragma unroll
  for (int k = 0; k + 1 < N; k += 2) {
    float2 s, c;
    sincos_turns2(th[k], th[k + 1], s, c);
    sn[k] = s.x;
    sn[k + 1] = s.y;
    cs[k] = c.x;
    cs[k + 1] = c.y;
  }
  if (N & 1) sincos_turns(th[N - 1], sn[N - 1], cs[N - 1]);
}

}  // namespace sde
