// josephson.cu -- per-path SRK2 integration of Eq. 1 on the GPU.
//
// Each path lives in registers for the whole launch (Alg. 1: load x, v and
// the parameters, loop over m steps, store back; Sec. 4.1).  One Philox
// block gives the Gaussians of four consecutive steps (Sec. 4.1 draws two
// uniforms per step; here one Gaussian per step suffices since Eq. 1 has one
// noise component).  The step is Alg. 2 applied to y = (x, v):
//
//   F1 = -gamma v - 2 pi cos(2 pi x) + a cos(omega t_n) + f
//   x~ = x + dt v,          v~ = v + dt F1 + s psi
//   F2 = -gamma v~ - 2 pi cos(2 pi x~) + a cos(omega t_{n+1}) + f
//   x' = x + dt/2 (v + v~), v' = v + dt/2 (F1 + F2) + s psi,   s = sqrt(2 gamma D dt)
//
// Time is kept modulo the drive period as the integer k = n mod P (Sec. 5),
// so cos(omega t_n) = cos(2 pi k / P) comes from a P-entry table in shared
// memory.  Position is kept as x in [0, 1) plus an integer winding count
// (folded once per group of four steps), so FP32 resolution does not degrade
// as paths run away.  cos(2 pi x) is a branch-free minimax polynomial
// (jj_force below).
//
// The window average of v (the time-averaged velocity <<v>> of Sec. 5) is
// summed in FP32 over blocks of 64 steps (aligned to absolute step indices)
// and flushed into an FP64 per-path accumulator; per-warp moments of the
// per-path averages are FP64.
//
// A thread advances one, two or four paths; with two or four, pairs of paths
// share Blackwell's packed FP32x2 FMA, add and multiply (jj_step2,
// box_muller_tab2), which round exactly like the scalar instructions, so
// every launch variant produces the same bits.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>
#include <string>

#include "internal.h"
#include "philox.cuh"

namespace sde {
namespace {

// A - 2 pi cos(2 pi x) for |x| < 2^22 without branches: with r = x - rint(x)
// in [-1/2, 1/2] and b = 1/4 - |r| in [-1/4, 1/4], cos(2 pi x) = sin(2 pi b),
// and sin(2 pi b) = b P(b^2) with P a degree-4 polynomial whose coefficients
// minimise the largest absolute error on [0, 1/4] (Lawson's iteratively
// reweighted least squares, about 3e-9 in exact arithmetic).  The factor
// -2 pi of Eq. 1's force is folded into P, so the force term and the addend
// A = a cos(omega t) + f - gamma v cost one FMA.  In FP32 the error of
// cos(2 pi x) is at most 1.7e-7 (RMS 3.7e-8).
__device__ __forceinline__ float jj_force(float x, float A) {
  const float b = 0.25f - fabsf(x - rintf(x));
  const float s = b * b;
  float p = -2.484164429e+02f;  // -2 pi x (39.536705, -76.5497818, 81.6010056, -41.3416557, 6.28318501)
  p = fmaf(p, s, 4.809764709e+02f);
  p = fmaf(p, s, -5.127142334e+02f);
  p = fmaf(p, s, 2.597572937e+02f);
  p = fmaf(p, s, -3.947841644e+01f);
  return fmaf(b, p, A);
}

// One SRK2 step (Alg. 2), or with EM one Euler-Maruyama step (the
// first-order scheme of PROG2, Sec. 4.2).  x is kept in [0, 1) up to the
// drift of the steps since the last wrap (at most four steps, see
// jj_segment).  e0, e1: the drive and bias a cos(omega t) + f at t_n and
// t_{n+1}.
template <bool ACC, bool EM>
__device__ __forceinline__ void jj_step(float &x, float &v, float &acc, float z, const JJConsts &c, float e0,
                                        float e1) {
  const float vn = fmaf(c.s, z, v);  // v plus the noise increment, used by both stages
  const float F1 = jj_force(x, fmaf(-c.gamma, v, e0));
  if (EM) {
    x = fmaf(c.dt, v, x);
    v = fmaf(c.dt, F1, vn);
    if (ACC) acc += v;
    return;
  }
  const float xt = fmaf(c.dt, v, x);
  const float vt = fmaf(c.dt, F1, vn);
  const float F2 = jj_force(xt, fmaf(-c.gamma, vt, e1));
  x = fmaf(c.h, v + vt, x);
  v = fmaf(c.h, F1 + F2, vn);
  if (ACC) acc += v;
}

// The same step for two paths at once on packed FP32 pairs (Blackwell's
// two-wide FMA, add and multiply, rounded like fmaf and +), so one
// instruction advances both paths of a thread.  Same operations in the same
// order as jj_force / jj_step: the results are bit-identical.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float2 jj_force2(float2 x, float2 A) {
  // -|r| by setting the sign bit; rint is symmetric, so -rint(x) = rint(-x)
  const float2 r = __fadd2_rn(x, make_float2(rintf(-x.x), rintf(-x.y)));
  const float2 nr = make_float2(__int_as_float(__float_as_int(r.x) | 0x80000000),
                                __int_as_float(__float_as_int(r.y) | 0x80000000));
  const float2 b = __fadd2_rn(f2(0.25f), nr);
  const float2 s = __fmul2_rn(b, b);
  float2 p = __ffma2_rn(f2(-2.484164429e+02f), s, f2(4.809764709e+02f));
  p = __ffma2_rn(p, s, f2(-5.127142334e+02f));
  p = __ffma2_rn(p, s, f2(2.597572937e+02f));
  p = __ffma2_rn(p, s, f2(-3.947841644e+01f));
  return __ffma2_rn(b, p, A);
}

template <bool ACC, bool EM>
__device__ __forceinline__ void jj_step2(float2 &x, float2 &v, float2 &acc, float2 z, const JJConsts &c, float e0,
                                         float e1) {
  const float2 vn = __ffma2_rn(f2(c.s), z, v);
  const float2 F1 = jj_force2(x, __ffma2_rn(f2(-c.gamma), v, f2(e0)));
  if (EM) {
    x = __ffma2_rn(f2(c.dt), v, x);
    v = __ffma2_rn(f2(c.dt), F1, vn);
    if (ACC) acc = __fadd2_rn(acc, v);
    return;
  }
  const float2 xt = __ffma2_rn(f2(c.dt), v, x);
  const float2 vt = __ffma2_rn(f2(c.dt), F1, vn);
  const float2 F2 = jj_force2(xt, __ffma2_rn(f2(-c.gamma), vt, f2(e1)));
  x = __ffma2_rn(f2(c.h), __fadd2_rn(v, vt), x);
  v = __ffma2_rn(f2(c.h), __fadd2_rn(F1, F2), vn);
  if (ACC) acc = __fadd2_rn(acc, v);
}

// Steps s of a group for all ILP paths (packed pairs where ILP is even).
template <int ILP, bool ACC, bool EM>
__device__ __forceinline__ void jj_steps(float (&x)[ILP], float (&v)[ILP], float (&acc)[ILP],
                                         const float (&z)[ILP][4], int s, const JJConsts &c, float e0, float e1) {
  if constexpr (ILP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < ILP; i += 2) {
      float2 X = make_float2(x[i], x[i + 1]), V = make_float2(v[i], v[i + 1]);
      float2 S = make_float2(acc[i], acc[i + 1]);
      jj_step2<ACC, EM>(X, V, S, make_float2(z[i][s], z[i + 1][s]), c, e0, e1);
      x[i] = X.x;
      x[i + 1] = X.y;
      v[i] = V.x;
      v[i + 1] = V.y;
      acc[i] = S.x;
      acc[i + 1] = S.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < ILP; ++i) jj_step<ACC, EM>(x[i], v[i], acc[i], z[i][s], c, e0, e1);
  }
}

// Fold x back into [0, 1), counting whole turns in w.
__device__ __forceinline__ void jj_wrap(float &x, int &w) {
  const float fl = floorf(x);
  x -= fl;
  w += (int)fl;
}

// Drive tables: the shared cos(2 pi k / P) table (P + 4 entries) and, for
// P <= kWarpTableMaxP, one table of a cos + f per warp, each padded to a
// multiple of 4 floats.
constexpr int kWarpTableMaxP = 1020;
constexpr int kJJMaxBlock = 512;  // the largest block any Josephson launch uses

__host__ __device__ inline int jj_table_stride(int P) { return (P + 4 + 3) & ~3; }

__host__ inline size_t jj_smem_bytes(int P, int block) {
  const int pp = jj_table_stride(P);
  return sizeof(float) * (size_t)pp * (P <= kWarpTableMaxP ? 1 + block / 32 : 1);
}

// The Box-Muller transforms of the Philox blocks r[i] of ILP paths into their
// four Gaussians z[i][0..3]: pairs of paths together on packed FP32 pairs
// (the same roundings as one path at a time), so each packed pair of paths
// gets its Gaussians already paired for jj_step2.
template <int ILP>
__device__ __forceinline__ void jj_transform(const uint4 (&r)[ILP], const float *bm_tab, float (&z)[ILP][4]) {
  if constexpr (ILP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < ILP; i += 2) {
      float2 Z0, Z1, Z2, Z3;
      box_muller_tab2(r[i].x, r[i].y, r[i + 1].x, r[i + 1].y, bm_tab, Z0, Z1);
      box_muller_tab2(r[i].z, r[i].w, r[i + 1].z, r[i + 1].w, bm_tab, Z2, Z3);
      z[i][0] = Z0.x;
      z[i + 1][0] = Z0.y;
      z[i][1] = Z1.x;
      z[i + 1][1] = Z1.y;
      z[i][2] = Z2.x;
      z[i + 1][2] = Z2.y;
      z[i][3] = Z3.x;
      z[i + 1][3] = Z3.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < ILP; ++i) {
      box_muller_tab(r[i].x, r[i].y, bm_tab, z[i][0], z[i][1]);
      box_muller_tab(r[i].z, r[i].w, bm_tab, z[i][2], z[i][3]);
    }
  }
}

// Advance ILP paths over the steps [n0, n1).  `k` is the drive-table index
// of step n0 (n0 mod P) and is updated.
// SCALED: `drive` holds a cos(2 pi k / P) + f for this point (a per-warp or
// per-point table), else cos(2 pi k / P) and the drive term is formed here.
template <int ILP, bool ACC, bool EM = false, bool SCALED = false, bool ONEBB = false>
__device__ __forceinline__ void jj_segment(float (&x)[ILP], int (&w)[ILP], float (&v)[ILP],
                                           double (&vs)[ILP], const JJConsts &c,
                                           const float *__restrict__ drive, int P, int &k,
                                           int64_t n0, int64_t n1, const PhiloxKeys &key,
                                           const uint32_t (&pid)[ILP], uint32_t point,
                                           const float *bm_tab) {
  if (n0 >= n1) return;
  float acc[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) acc[i] = 0.0f;
  // group indices fit in 32 bits: steps are at most 2^33
  const uint32_t g0 = (uint32_t)(n0 >> 2), g1 = (uint32_t)((n1 - 1) >> 2);
  // Blocks of 16 groups (64 steps) aligned to absolute step indices; the
  // FP32 partial sums are flushed after each block, outside the group loop,
  // so the FP64 adds run once per 64 steps.
  // PIPE (four or more paths per thread): the Gaussians of group g + 1 are
  // drawn while group g is stepped, in one basic block, so the integer Philox
  // work interleaves with the FP32 steps (16 more live registers; with fewer
  // paths per thread the lost occupancy costs more than the overlap gains).
  constexpr bool PIPE = ILP >= 4;  // with ONEBB (the four-path kernels): see the group loop
  float z[ILP][4];
  if constexpr (PIPE) {
    uint4 r0[ILP];
#pragma unroll
    for (int i = 0; i < ILP; ++i) r0[i] = philox4x32_10(make_uint4(g0, pid[i], point, kTagJosephson), key);
    jj_transform<ILP>(r0, bm_tab, z);
  }
  for (uint32_t gb = g0; gb <= g1; gb = (gb | 15u) + 1u) {
    const uint32_t ge = (gb | 15u) < g1 ? (gb | 15u) : g1;
    for (uint32_t g = gb; g <= ge; ++g) {
      if constexpr (PIPE && ONEBB) {
        // ONEBB: a whole group with P a multiple of 4 as one basic block --
        // the next group's Philox words, the four steps, the position fold
        // and the next group's Box-Muller transform -- so that the compiler
        // can interleave the integer, special-function and FP32 work of
        // all three (the same operations as below, in the same order per
        // value: bit-identical).
        const int64_t base = (int64_t)g << 2;
        if ((P & 3) == 0 && base >= n0 && base + 4 <= n1) {
          uint4 rn[ILP];
#pragma unroll
          for (int i = 0; i < ILP; ++i)
            rn[i] = philox4x32_10(make_uint4(g + 1, pid[i], point, kTagJosephson), key);
          const float4 d = *reinterpret_cast<const float4 *>(drive + k);
          const float d4 = drive[k + 4];
          float e[5];
          e[0] = SCALED ? d.x : fmaf(c.a, d.x, c.f);
          e[1] = SCALED ? d.y : fmaf(c.a, d.y, c.f);
          e[2] = SCALED ? d.z : fmaf(c.a, d.z, c.f);
          e[3] = SCALED ? d.w : fmaf(c.a, d.w, c.f);
          e[4] = SCALED ? d4 : fmaf(c.a, d4, c.f);
          k = (k + 4 == P) ? 0 : k + 4;
#pragma unroll
          for (int s = 0; s < 4; ++s) jj_steps<ILP, ACC, EM>(x, v, acc, z, s, c, e[s], e[s + 1]);
#pragma unroll
          for (int i = 0; i < ILP; ++i) jj_wrap(x[i], w[i]);
          jj_transform<ILP>(rn, bm_tab, z);
          continue;
        }
      }
      // PIPE: the Philox words of group g + 1 now, their Box-Muller
      // transform into z once this group's steps have read it
      uint4 rn[ILP];
#pragma unroll
      for (int i = 0; i < ILP; ++i)
        rn[i] = philox4x32_10(make_uint4(PIPE ? g + 1 : g, pid[i], point, kTagJosephson), key);
      if constexpr (!PIPE) jj_transform<ILP>(rn, bm_tab, z);
      const int64_t base = (int64_t)g << 2;
      if (base >= n0 && base + 4 <= n1) {
        // full group: drive values at t_{4g} .. t_{4g+4}
        float e[5];
        if ((P & 3) == 0) {
          // k is a multiple of 4 here; the table is padded by 4 entries
          const float4 d = *reinterpret_cast<const float4 *>(drive + k);
          e[0] = SCALED ? d.x : fmaf(c.a, d.x, c.f);
          e[1] = SCALED ? d.y : fmaf(c.a, d.y, c.f);
          e[2] = SCALED ? d.z : fmaf(c.a, d.z, c.f);
          e[3] = SCALED ? d.w : fmaf(c.a, d.w, c.f);
          e[4] = SCALED ? drive[k + 4] : fmaf(c.a, drive[k + 4], c.f);
          k += 4;
          if (k == P) k = 0;
        } else {
#pragma unroll
          for (int s = 0; s < 5; ++s) {
            e[s] = SCALED ? drive[k] : fmaf(c.a, drive[k], c.f);
            if (s < 4) k = (k + 1 == P) ? 0 : k + 1;
          }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) jj_steps<ILP, ACC, EM>(x, v, acc, z, s, c, e[s], e[s + 1]);
      } else {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const int64_t n = base + s;
          if (n >= n0 && n < n1) {
            const float e0 = SCALED ? drive[k] : fmaf(c.a, drive[k], c.f);
            k = (k + 1 == P) ? 0 : k + 1;
            const float e1 = SCALED ? drive[k] : fmaf(c.a, drive[k], c.f);
            jj_steps<ILP, ACC, EM>(x, v, acc, z, s, c, e0, e1);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < ILP; ++i) jj_wrap(x[i], w[i]);
      if constexpr (PIPE) jj_transform<ILP>(rn, bm_tab, z);
    }
    // Flush the FP32 partial sums at absolute 64-step boundaries, so that a
    // run split at any multiple of 64 steps reproduces the unsplit sums.
    if (ACC && ((ge + 1) & 15) == 0) {
#pragma unroll
      for (int i = 0; i < ILP; ++i) {
        vs[i] += (double)acc[i];
        acc[i] = 0.0f;
      }
    }
  }
  if (ACC) {
#pragma unroll
    for (int i = 0; i < ILP; ++i) vs[i] += (double)acc[i];
  }
}

__device__ __forceinline__ double warp_sum(double a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  return a;
}

template <int ILP, bool EM, bool ONEBB = false>
__device__ __forceinline__ void jj_unit(const JJLaunchArgs &A, int u, const float *drive, float *wtab,
                                        const float *bm_tab, int lane) {
  const JJUnit un = A.units[u];
  const JJConsts c = A.consts[un.point];
  const PhiloxKeys &key = A.keys;
  float x[ILP], v[ILP];
  int w[ILP];
  double vs[ILP];
  uint32_t pid[ILP];
  bool valid[ILP];
  int64_t gi[ILP];
#pragma unroll
  for (int i = 0; i < ILP; ++i) {
    const int j = lane + 32 * i;
    valid[i] = j < un.n_paths;
    pid[i] = (uint32_t)(un.path_begin + j);
    gi[i] = c.path_offset + un.path_begin + j;
    x[i] = 0.0f;
    v[i] = 0.0f;
    w[i] = 0;
    vs[i] = 0.0;
    if (valid[i]) {
      x[i] = A.st.x_in[gi[i]];
      v[i] = A.st.v_in[gi[i]];
      if (A.st.w_in) w[i] = A.st.w_in[gi[i]];
      if (A.st.vsum_in) vs[i] = A.st.vsum_in[gi[i]];
    }
    const float fl = floorf(x[i]);
    x[i] -= fl;
    w[i] += (int)fl;
  }
  const int64_t nb = A.n_begin;
  const int64_t ne = A.n_end < c.steps ? A.n_end : c.steps;
  if (nb < ne) {
    int k = (int)(nb % A.P);
    const int64_t split = ne < c.wstart ? ne : c.wstart;
    const int64_t w0 = nb > c.wstart ? nb : c.wstart;
    if (wtab) {
      // this warp's copy of the drive term a cos(2 pi k / P) + f of the unit's point
      for (int q = lane; q < A.P + 4; q += 32) wtab[q] = fmaf(c.a, drive[q], c.f);
      __syncwarp();
      jj_segment<ILP, false, EM, true, ONEBB>(x, w, v, vs, c, wtab, A.P, k, nb, split, key, pid,
                                              (uint32_t)un.point, bm_tab);
      jj_segment<ILP, true, EM, true, ONEBB>(x, w, v, vs, c, wtab, A.P, k, w0, ne, key, pid, (uint32_t)un.point,
                                             bm_tab);
      __syncwarp();  // the table is rewritten for the warp's next unit
    } else {
      jj_segment<ILP, false, EM, false, ONEBB>(x, w, v, vs, c, drive, A.P, k, nb, split, key, pid,
                                               (uint32_t)un.point, bm_tab);
      jj_segment<ILP, true, EM, false, ONEBB>(x, w, v, vs, c, drive, A.P, k, w0, ne, key, pid, (uint32_t)un.point,
                                              bm_tab);
    }
  }
  bool bad = false;
#pragma unroll
  for (int i = 0; i < ILP; ++i) {
    if (valid[i]) {
      A.st.x_out[gi[i]] = x[i];
      A.st.v_out[gi[i]] = v[i];
      A.st.w_out[gi[i]] = w[i];
      A.st.vsum_out[gi[i]] = vs[i];
      bad |= !(isfinite(x[i]) && isfinite(v[i]));
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(A.err, kErrNonFinite);

  // Moments of the per-path window averages of this unit.
  const int64_t reach = A.n_end < c.steps ? A.n_end : c.steps;
  const int64_t wcount = reach > c.wstart ? reach - c.wstart : 0;
  double cnt = 0.0, sum = 0.0;
  if (wcount > 0) {
#pragma unroll
    for (int i = 0; i < ILP; ++i)
      if (valid[i]) {
        cnt += 1.0;
        sum += vs[i] / (double)wcount;
      }
  }
  cnt = warp_sum(cnt);
  sum = warp_sum(sum);
  const double mean = cnt > 0.0 ? sum / cnt : 0.0;
  double m2 = 0.0;
  if (wcount > 0) {
#pragma unroll
    for (int i = 0; i < ILP; ++i)
      if (valid[i]) {
        const double d = vs[i] / (double)wcount - mean;
        m2 += d * d;
      }
  }
  m2 = warp_sum(m2);
  if (lane == 0) A.partials[u] = Moments{cnt, mean, m2};
}

template <int ILP, bool EM, bool ONEBB = false>
__device__ __forceinline__ void jj_kernel_body(const JJLaunchArgs &A) {
  // drive table cos(2 pi k / P), k = 0 .. P + 3 (four entries of padding
  // repeat the start of the period), 16-byte aligned
  extern __shared__ float4 drive_s4[];
  __shared__ float bm_tab[2 * kBmTable];  // Box-Muller angle table
  float *drive_s = reinterpret_cast<float *>(drive_s4);
  for (int i = threadIdx.x; i < A.P + 4; i += blockDim.x) drive_s[i] = A.drive[i % A.P];
  fill_bm_table(bm_tab);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  // per-warp tables of the drive term (P <= kWarpTableMaxP), 16-byte aligned
  const int pp = jj_table_stride(A.P);
  float *wtab = A.P <= kWarpTableMaxP ? drive_s + pp * (1 + (threadIdx.x >> 5)) : nullptr;
  if (A.queue) {
    // Persistent: warps pull units from the longest-first work list.
    for (;;) {
      int u = 0;
      if (lane == 0) u = (int)atomicAdd(A.queue, 1u) + A.unit_begin;
      u = __shfl_sync(0xffffffffu, u, 0);
      if (u >= A.unit_end) break;
      jj_unit<ILP, EM, ONEBB>(A, u, drive_s, wtab, bm_tab, lane);
    }
  } else {
    const int u = A.unit_begin + blockIdx.x * warps + (threadIdx.x >> 5);
    if (u < A.unit_end) jj_unit<ILP, EM, ONEBB>(A, u, drive_s, wtab, bm_tab, lane);
  }
}

template <int ILP, bool EM = false>
__global__ void __launch_bounds__(512) jj_kernel(const JJLaunchArgs A) {
  jj_kernel_body<ILP, EM>(A);
}

// The same kernel with registers capped at 64 per thread (blocks of up to 512
// threads, two per SM): more resident warps for more spills; the autotuner
// picks.
template <int ILP, bool EM = false>
__global__ void __launch_bounds__(512, 2) jj_kernel_cap64(const JJLaunchArgs A) {
  jj_kernel_body<ILP, EM>(A);
}

// Packed-pair kernels (2 or 4 paths per thread) at the fewest registers that
// hold them without spills: 72 for one pair (28 warps per SM in blocks of
// 128), 128 for two pairs with the noise of the next group in flight (16
// warps, each with two independent pairs and the Philox work to overlap).
template <int ILP, bool EM = false>
__global__ void __maxnreg__(ILP == 2 ? 72 : 128) jj_kernel_packed(const JJLaunchArgs A) {
  jj_kernel_body<ILP, EM, ILP >= 4>(A);
}

// Four paths per thread held to 96 registers (20 warps per SM in blocks of
// 128): the autotuner weighs the extra warps against the compiler's freedom
// to overlap.
template <bool EM = false>
__global__ void __maxnreg__(96) jj_kernel_packed4_cap96(const JJLaunchArgs A) {
  jj_kernel_body<4, EM, true>(A);
}

__global__ void jj_prepare_kernel(const sde_jj_point *pts, int n_points, int P,
                                  const int64_t *steps, const int64_t *offsets,
                                  const int64_t *paths, JJConsts *out, float *drive) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_points) {
    const sde_jj_point p = pts[t];
    const double dt = 2.0 * 3.14159265358979323846 / (p.omega * (double)P);
    JJConsts c;
    c.gamma = (float)p.gamma;
    c.a = (float)p.a;
    c.f = (float)p.f;
    c.dt = (float)dt;
    c.h = (float)(0.5 * dt);
    c.s = (float)sqrt(2.0 * p.gamma * p.D * dt);
    c.paths = (int32_t)paths[t];
    c.pad = 0;
    c.steps = steps[t];
    c.wstart = steps[t] - steps[t] / 2;
    c.path_offset = offsets[t];
    c.dt64 = dt;
    out[t] = c;
  }
  if (t < P) drive[t] = (float)cospi(2.0 * (double)t / (double)P);
}

// Merge of two (n, mean, M2) triples (Chan, Golub & LeVeque 1979).
__device__ __forceinline__ Moments merge(const Moments &a, const Moments &b) {
  const double n = a.n + b.n;
  if (n == 0.0) return Moments{0.0, 0.0, 0.0};
  const double d = b.mean - a.mean;
  return Moments{n, a.mean + d * (b.n / n), a.m2 + b.m2 + d * d * (a.n * b.n / n)};
}

// One warp per point: lane-strided merge over the point's units in a fixed
// order, then a fixed shuffle tree (deterministic result).
__global__ void jj_finalize_kernel(const JJConsts *consts, const int2 *range, int n_points,
                                   const Moments *partials, int64_t n_end, sde_obs_row *obs) {
  const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= n_points) return;
  const int2 r = range[p];
  Moments m{0.0, 0.0, 0.0};
  for (int u = r.x + lane; u < r.y; u += 32) m = merge(m, partials[u]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Moments q;
    q.n = __shfl_down_sync(0xffffffffu, m.n, o);
    q.mean = __shfl_down_sync(0xffffffffu, m.mean, o);
    q.m2 = __shfl_down_sync(0xffffffffu, m.m2, o);
    if (lane + o < 32) m = merge(m, q);
  }
  if (lane == 0) {
    const JJConsts c = consts[p];
    const int64_t reach = n_end < c.steps ? n_end : c.steps;
    sde_obs_row row;
    row.count = m.n;
    row.mean = m.n > 0.0 ? m.mean : 0.0;
    row.var = m.n > 1.0 ? m.m2 / (m.n - 1.0) : 0.0;
    row.se = m.n > 0.0 ? sqrt(row.var / m.n) : 0.0;
    row.t = (double)reach * c.dt64;
    obs[p] = row;
  }
}

__global__ void philox_fill_kernel(const uint4 *ctr, uint2 key, uint4 *out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = philox4x32_10(ctr[i], key);
}

__global__ void box_muller_fill_kernel(const uint4 *ctr, uint2 key, float4 *z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox4x32_10(ctr[i], key);
    float4 o;
    box_muller(r.x, r.y, o.x, o.y);
    box_muller(r.z, r.w, o.z, o.w);
    z[i] = o;
  }
}

// Box-Muller of given word pairs (w0, w1) -> (z0, z1): variant 0 the
// library's default transform, 1 the Josephson kernels' (table angle,
// hardware logarithm).
__global__ void box_muller_words_kernel(const uint2 *w, int64_t n, int variant, float2 *z) {
  __shared__ float tab[2 * kBmTable];
  fill_bm_table(tab);
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint2 p = w[i];
    float2 o;
    if (variant == 1)
      box_muller_tab(p.x, p.y, tab, o.x, o.y);
    else
      box_muller(p.x, p.y, o.x, o.y);
    z[i] = o;
  }
}

void *jj_kernel_ptr(int variant) {
  switch (variant) {
    case 1: return (void *)jj_kernel<1>;
    case 2: return (void *)jj_kernel_packed<2>;
    case 4: return (void *)jj_kernel_packed<4>;
    case 14: return (void *)jj_kernel_packed4_cap96<>;
    case 11: return (void *)jj_kernel_cap64<1>;
    case 12: return (void *)jj_kernel_cap64<2>;
    case 101: return (void *)jj_kernel<1, true>;
    case 102: return (void *)jj_kernel_packed<2, true>;
    case 104: return (void *)jj_kernel_packed<4, true>;
    case 111: return (void *)jj_kernel_cap64<1, true>;
    case 112: return (void *)jj_kernel_cap64<2, true>;
    case 114: return (void *)jj_kernel_packed4_cap96<true>;
  }
  return nullptr;
}

}  // namespace

cudaError_t jj_prepare(const sde_jj_point *points_dev, int n_points, int P, const int64_t *steps_dev,
                       const int64_t *offsets_dev, const int64_t *paths_dev, JJConsts *consts_dev,
                       float *drive_dev, cudaStream_t s) {
  const int n = n_points > P ? n_points : P;
  jj_prepare_kernel<<<(n + 255) / 256, 256, 0, s>>>(points_dev, n_points, P, steps_dev, offsets_dev,
                                                    paths_dev, consts_dev, drive_dev);
  return cudaGetLastError();
}

// `ilp` encodes the variant: 1, 2, 4 = paths per thread; +10 = fewer registers
// (64 for 1 and 2 paths per thread, 96 for 4); +100 = Euler-Maruyama.
cudaError_t jj_launch(const JJLaunchArgs &a, int ilp, int block, int grid, cudaStream_t s) {
  const size_t smem = jj_smem_bytes(a.P, block);
  switch (ilp) {
    case 1: jj_kernel<1><<<grid, block, smem, s>>>(a); break;
    case 2: jj_kernel_packed<2><<<grid, block, smem, s>>>(a); break;
    case 4: jj_kernel_packed<4><<<grid, block, smem, s>>>(a); break;
    case 14: jj_kernel_packed4_cap96<><<<grid, block, smem, s>>>(a); break;
    case 11: jj_kernel_cap64<1><<<grid, block, smem, s>>>(a); break;
    case 12: jj_kernel_cap64<2><<<grid, block, smem, s>>>(a); break;
    // Euler-Maruyama variants: the code + 100
    case 101: jj_kernel<1, true><<<grid, block, smem, s>>>(a); break;
    case 102: jj_kernel_packed<2, true><<<grid, block, smem, s>>>(a); break;
    case 104: jj_kernel_packed<4, true><<<grid, block, smem, s>>>(a); break;
    case 111: jj_kernel_cap64<1, true><<<grid, block, smem, s>>>(a); break;
    case 112: jj_kernel_cap64<2, true><<<grid, block, smem, s>>>(a); break;
    case 114: jj_kernel_packed4_cap96<true><<<grid, block, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int jj_max_blocks_per_sm(int ilp, int block, int P) {
  int nb = 0;
  void *k = jj_kernel_ptr(ilp);
  if (!k) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, jj_smem_bytes(P, block)) != cudaSuccess)
    return 0;
  return nb;
}

// The dynamic shared memory limit is a per-function maximum shared by every
// launch in the process, so it is raised once, to what the largest table
// layout (P = kWarpTableMaxP, kJJMaxBlock threads) needs, and never lowered.
cudaError_t jj_configure() {
  static const cudaError_t status = [] {
    const int smem = (int)jj_smem_bytes(kWarpTableMaxP, kJJMaxBlock);
    const int variants[] = {1, 2, 4, 11, 12, 14, 101, 102, 104, 111, 112, 114};
    for (int v : variants) {
      const cudaError_t e = cudaFuncSetAttribute(jj_kernel_ptr(v), cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }();
  return status;
}

cudaError_t jj_finalize(const JJConsts *consts, const int2 *point_range, int n_points,
                        const Moments *partials, int64_t n_end, sde_obs_row *obs, cudaStream_t s) {
  const int wpb = 8;
  jj_finalize_kernel<<<(n_points + wpb - 1) / wpb, 32 * wpb, 0, s>>>(consts, point_range, n_points,
                                                                    partials, n_end, obs);
  return cudaGetLastError();
}

cudaError_t philox_fill(const uint32_t *ctr, uint64_t seed, uint32_t *out, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  philox_fill_kernel<<<(int)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(
      (const uint4 *)ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), (uint4 *)out, n);
  return cudaGetLastError();
}

cudaError_t box_muller_fill(const uint32_t *ctr, uint64_t seed, float *z, int64_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  box_muller_fill_kernel<<<(int)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(
      (const uint4 *)ctr, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), (float4 *)z, n);
  return cudaGetLastError();
}

cudaError_t box_muller_words(const uint32_t *w, int64_t n, int variant, float *z, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  box_muller_words_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>((const uint2 *)w, n, variant,
                                                                               (float2 *)z);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the per-path kernel (sde_josephson_run_noalloc).
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or arena (which forbids allocations behind its
// back), code that is itself being captured into a CUDA graph by a host
// program, or embedded/real-time hosts that pre-reserve all device memory at
// start-up.  For them this entry point keeps its only scratch -- one
// reduction partial per warp of 32 paths -- in a fixed array in the
// library's static device memory instead of a workspace allocated by
// sde_create.  Every GPU that loads the library holds this array until the
// process exits.
// ---------------------------------------------------------------------------

#define SDE_NOALLOC_UNITS (SDE_NOALLOC_MAX_PATHS / 32)

namespace {

// 32768 partials x 24 bytes = 768 KiB.  Shared by every call on a device;
// it keeps the previous call's contents.  Each call writes every slot it
// later reads, so nothing has to be cleared first.
static __device__ __align__(256) Moments g_noalloc_partials[SDE_NOALLOC_UNITS];

struct NoallocArgs {
  sde_jj_point p;
  int32_t P;
  int32_t n_paths;
  int64_t steps;
  int64_t n_begin, n_end;
  uint64_t seed;
  PhiloxKeys keys;
  JJState st;
  Moments *partials;  // device address of g_noalloc_partials
};

// One warp per 32 paths, one path per thread: the same arithmetic and the same
// unit decomposition as the plain schedule with one path per thread.
__global__ void __launch_bounds__(256) jj_noalloc_kernel(const NoallocArgs A) {
  extern __shared__ float4 drive_s4[];
  __shared__ float bm_tab[2 * kBmTable];
  float *drive_s = reinterpret_cast<float *>(drive_s4);
  const double dt = 2.0 * 3.14159265358979323846 / (A.p.omega * (double)A.P);
  for (int i = threadIdx.x; i < A.P + 4; i += blockDim.x)
    drive_s[i] = (float)cospi(2.0 * (double)(i % A.P) / (double)A.P);
  fill_bm_table(bm_tab);
  __syncthreads();
  JJConsts c;
  c.gamma = (float)A.p.gamma;
  c.a = (float)A.p.a;
  c.f = (float)A.p.f;
  c.dt = (float)dt;
  c.h = (float)(0.5 * dt);
  c.s = (float)sqrt(2.0 * A.p.gamma * A.p.D * dt);
  c.paths = A.n_paths;
  c.pad = 0;
  c.steps = A.steps;
  c.wstart = A.steps - A.steps / 2;
  c.path_offset = 0;
  c.dt64 = dt;
  const int u = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int n_units = (A.n_paths + 31) / 32;
  if (u >= n_units) return;
  const int lane = threadIdx.x & 31;
  const PhiloxKeys &key = A.keys;
  const int j = u * 32 + lane;
  const bool valid = j < A.n_paths;
  float x[1] = {0.0f}, v[1] = {0.0f};
  int w[1] = {0};
  double vs[1] = {0.0};
  const uint32_t pid[1] = {(uint32_t)j};
  if (valid) {
    x[0] = A.st.x_in[j];
    v[0] = A.st.v_in[j];
    if (A.st.w_in) w[0] = A.st.w_in[j];
    if (A.st.vsum_in) vs[0] = A.st.vsum_in[j];
  }
  const float fl = floorf(x[0]);
  x[0] -= fl;
  w[0] += (int)fl;
  const int64_t ne = A.n_end < c.steps ? A.n_end : c.steps;
  if (A.n_begin < ne) {
    int k = (int)(A.n_begin % A.P);
    const int64_t split = ne < c.wstart ? ne : c.wstart;
    jj_segment<1, false>(x, w, v, vs, c, drive_s, A.P, k, A.n_begin, split, key, pid, 0u, bm_tab);
    jj_segment<1, true>(x, w, v, vs, c, drive_s, A.P, k, A.n_begin > c.wstart ? A.n_begin : c.wstart, ne,
                        key, pid, 0u, bm_tab);
  }
  if (valid) {
    A.st.x_out[j] = x[0];
    A.st.v_out[j] = v[0];
    A.st.w_out[j] = w[0];
    A.st.vsum_out[j] = vs[0];
  }
  const int64_t wcount = ne > c.wstart ? ne - c.wstart : 0;
  const double m = (valid && wcount > 0) ? vs[0] / (double)wcount : 0.0;
  const double cnt = warp_sum((valid && wcount > 0) ? 1.0 : 0.0);
  const double mean = cnt > 0.0 ? warp_sum(m) / cnt : 0.0;
  const double d = (valid && wcount > 0) ? m - mean : 0.0;
  const double m2 = warp_sum(d * d);
  if (lane == 0) A.partials[u] = Moments{cnt, mean, m2};
}

__global__ void jj_noalloc_finalize(const Moments *partials, int n_units, int64_t steps, double dt,
                                    int64_t n_end, sde_obs_row *obs) {
  const int lane = threadIdx.x & 31;
  Moments m{0.0, 0.0, 0.0};
  for (int u = lane; u < n_units; u += 32) m = merge(m, partials[u]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Moments q;
    q.n = __shfl_down_sync(0xffffffffu, m.n, o);
    q.mean = __shfl_down_sync(0xffffffffu, m.mean, o);
    q.m2 = __shfl_down_sync(0xffffffffu, m.m2, o);
    if (lane + o < 32) m = merge(m, q);
  }
  if (lane == 0) {
    const int64_t reach = n_end < steps ? n_end : steps;
    sde_obs_row row;
    row.count = m.n;
    row.mean = m.n > 0.0 ? m.mean : 0.0;
    row.var = m.n > 1.0 ? m.m2 / (m.n - 1.0) : 0.0;
    row.se = m.n > 0.0 ? sqrt(row.var / m.n) : 0.0;
    row.t = (double)reach * dt;
    *obs = row;
  }
}

}  // namespace

namespace {
// Device address of g_noalloc_partials, resolved once per device.
constexpr int kMaxDevices = 64;
Moments *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;
}  // namespace

}  // namespace sde

extern "C" sde_status sde_josephson_run_noalloc(const sde_jj_point *point, int32_t steps_per_period,
                                                int64_t n_paths, int64_t total_steps, uint64_t seed,
                                                int64_t n_begin, int64_t n_end, const float *x_in_dev,
                                                const float *v_in_dev, const int32_t *w_in_dev,
                                                const double *vsum_in_dev, float *x_out_dev,
                                                float *v_out_dev, int32_t *w_out_dev,
                                                double *vsum_out_dev, sde_obs_row *obs_dev,
                                                void *stream) {
  using namespace sde;
  clear_error();
  SDE_CHECK_ARG(point != nullptr, "point is NULL");
  SDE_CHECK_ARG(n_paths >= 0, "n_paths must be >= 0");
  if (n_paths > SDE_NOALLOC_MAX_PATHS) {
    set_error("invalid argument: sde_josephson_run_noalloc handles at most " +
              std::to_string(SDE_NOALLOC_MAX_PATHS) + " paths per call (got " +
              std::to_string(n_paths) + "); use sde_create/sde_run_ensemble for larger ensembles");
    return SDE_ERR_INVALID_ARG;
  }
  SDE_CHECK_ARG(steps_per_period >= 1 && steps_per_period <= 4096, "steps_per_period must be in [1, 4096]");
  SDE_CHECK_ARG(total_steps >= 0 && total_steps <= (1ll << 33), "total_steps out of range");
  SDE_CHECK_ARG(n_begin >= 0 && n_end >= n_begin && n_end <= (1ll << 33), "need 0 <= n_begin <= n_end");
  SDE_CHECK_ARG(isfinite(point->gamma) && isfinite(point->a) && isfinite(point->omega) &&
                    isfinite(point->f) && isfinite(point->D),
                "point parameters must be finite");
  SDE_CHECK_ARG(point->omega > 0.0 && point->gamma > 0.0 && point->D >= 0.0,
                "need omega > 0, gamma > 0, D >= 0");
  SDE_CHECK_ARG(obs_dev != nullptr, "obs_dev is NULL");
  if (n_paths > 0)
    SDE_CHECK_ARG(x_in_dev && v_in_dev && x_out_dev && v_out_dev && w_out_dev && vsum_out_dev,
                  "x_in, v_in, x_out, v_out, w_out and vsum_out must be non-NULL");
  int dev = 0;
  SDE_CUDA_TRY(cudaGetDevice(&dev));
  SDE_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device index out of range");
  Moments *partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
      g_noalloc_ptr[dev] = (Moments *)p;
    }
    partials = g_noalloc_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  NoallocArgs a{};
  a.p = *point;
  a.P = steps_per_period;
  a.n_paths = (int32_t)n_paths;
  a.steps = total_steps;
  a.n_begin = n_begin;
  a.n_end = n_end;
  a.seed = seed;
  a.keys = philox_round_keys(seed);
  a.st = JJState{x_in_dev, v_in_dev, w_in_dev, vsum_in_dev, x_out_dev, v_out_dev, w_out_dev, vsum_out_dev};
  a.partials = partials;
  const int n_units = (int)((n_paths + 31) / 32);
  if (n_units > 0) {
    jj_noalloc_kernel<<<(n_units + 7) / 8, 256, sizeof(float) * (steps_per_period + 4), s>>>(a);
    SDE_CUDA_TRY(cudaGetLastError());
  }
  const double dt = 2.0 * 3.14159265358979323846 / (point->omega * (double)steps_per_period);
  jj_noalloc_finalize<<<1, 32, 0, s>>>(partials, n_units, total_steps, dt, n_end, obs_dev);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}
