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

}  // namespace sde
