// kuramoto.cu -- SRK2 integration of the noisy Kuramoto model (Eq. 2,
// gamma = 1) on the GPU, in three forms of the coupling sum:
//
//  * mean field (Eq. 3): sum_j sin(x_j - x_i) = cos x_i S - sin x_i C with
//    S = sum_j sin x_j, C = sum_j cos x_j.  One CTA owns one replica for the
//    whole run: its phases stay in registers, S and C come from a block
//    reduction per stage (two per step), r(t) = sqrt(S^2 + C^2) / N is read
//    off the first-stage sums.  No grid-wide synchronisation.
//  * mean field over the whole grid (Eq. 3 for replicas too large for a CTA
//    or a cluster, such as the 2^24 oscillators of Fig. 4): two launches
//    per step, each reducing its partial sums of sin/cos through the last
//    block to finish (fixed-order FP64 sum of the per-block partials, no
//    waiting between blocks).
//  * pairwise (Alg. 3 / Fig. 3): the direct all-pairs sum, tiles of source
//    phases staged in shared memory; one launch per SRK2 stage with the
//    sub-step fused into the epilogue (Sec. 4.2 splits it into UpdateRHS and
//    AdvanceSystem; higher order by interleaving stages).
//  * general K_ij: the sum as a GEMM against [sin x | cos x] (see
//    kuramoto_general.cu).
//
// Phases are kept as 32-bit fixed-point turns (2^32 units per 2 pi): the
// wrap modulo 2 pi is exact integer overflow and the resolution (1.5e-9
// rad) does not depend on the phase, in the spirit of keeping time modulo
// the period (Sec. 5).  Drift increments are computed in FP32 and rounded to
// the fixed-point grid once per stage (the predictor phase too), and sin/cos
// of a phase come from its fixed-point value directly (turns.cuh).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cooperative_groups.h>

#include "kuramoto.h"
#include "kuramoto_internal.h"
#include "philox.cuh"
#include "turns.cuh"

namespace sde {

namespace {

__device__ __forceinline__ float2 warp_sum2(float a, float b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  return make_float2(a, b);
}

// Sum of (a, b) over the block; every thread receives the totals.  `red`
// alternates between two slots so one barrier per reduction suffices.
__device__ __forceinline__ float2 block_sum2(float a, float b, float2 *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 v = warp_sum2(a, b);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = lane < nw ? red[lane] : make_float2(0.0f, 0.0f);
  return warp_sum2(v.x, v.y);
}

// Partial sums of sin and cos in fixed point, units of 2^-17 (the replica
// forms that keep a replica in one CTA or cluster, n_osc <= 8192): integer
// sums are exact and associative, so the totals are the same however the
// oscillators are split over threads, warps and CTAs, and a warp adds 32
// values in one redux instruction.  |sum| <= 8192 x 2^17 = 2^30.  The
// quantisation (<= 2^-18 per value) moves S and C by ~1e-5 at N = 4096,
// which reaches a phase only through K dt / (2 pi N).
constexpr float kQuant = 131072.0f;
constexpr float kInvQuant = 1.0f / 131072.0f;

// round(v 2^17) to the nearest integer (ties to even) for |v| <= 1, on the FMA
// pipe: v 2^17 + 1.5 2^23 lies in [2^23, 2^24), where the FP32 spacing is 1,
// so the one rounding of the FMA is the rounding to an integer, read off the
// mantissa bits.  The same integer as __float2int_rn(v * 2^17), without the
// conversion unit.
__device__ __forceinline__ int quant(float v) {
  return __float_as_int(fmaf(v, kQuant, 12582912.0f)) - 0x4B400000;
}

__device__ __forceinline__ int2 warp_qsum(int a, int b) {
  return make_int2(__reduce_add_sync(0xffffffffu, a), __reduce_add_sync(0xffffffffu, b));
}

__device__ __forceinline__ float2 unquant(int2 v) { return make_float2((float)v.x * kInvQuant, (float)v.y * kInvQuant); }

// Block total of the fixed-point pair; every thread receives it.  `red`
// alternates between two slots so one barrier per reduction suffices.
__device__ __forceinline__ float2 block_qsum(int a, int b, int2 *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int2 v = warp_qsum(a, b);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  v = lane < nw ? red[lane] : make_int2(0, 0);
  return unquant(warp_qsum(v.x, v.y));
}

// Blocks of up to 1024 threads hold 1-2 oscillators per thread; larger
// per-thread counts run in blocks of at most 512 threads (128 registers).
template <int OPT>
__global__ void __launch_bounds__(OPT <= 2 ? 1024 : 512, 1) kur_meanfield_kernel(const KurArgs A) {
  __shared__ int2 red[2][32];
  const int rep = blockIdx.x;
  const int64_t N = A.N;
  const int64_t base = (int64_t)rep * N;
  const uint2 key = seed_to_key(A.seed);
  uint32_t th[OPT];
  float wdt[OPT];
  bool valid[OPT];
#pragma unroll
  for (int k = 0; k < OPT; ++k) {
    const int64_t i = threadIdx.x + (int64_t)k * blockDim.x;
    valid[k] = i < N;
    th[k] = valid[k] ? A.theta_in[base + i] : 0u;
    wdt[k] = valid[k] ? A.omega[base + i] * A.wscale : 0.0f;
  }
  int slot = 0;
  int64_t sample_ctr = 0;  // (n - n_begin) mod M
  int64_t sample_idx = 0;
  const float invN = 1.0f / (float)N;
  for (int64_t n = A.n_begin; n < A.n_end;) {
    const int64_t g = n >> 2;
    float z[OPT][4];
#pragma unroll
    for (int k = 0; k < OPT; ++k)
      gauss4((uint32_t)g, (uint32_t)(threadIdx.x + k * blockDim.x), (uint32_t)rep, kTagKuramoto, key,
             z[k]);
    const int s0 = (int)(n & 3);
    const int64_t rem = A.n_end - (g << 2);
    const int s1 = rem < 4 ? (int)rem : 4;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s < s0 || s >= s1) continue;
      float sn[OPT], cs[OPT];
      int S = 0, C = 0;
      sincos_turns_n<OPT>(th, sn, cs);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn[k] = cs[k] = 0.0f;
        S += quant(sn[k]);
        C += quant(cs[k]);
      }
      float2 sc = block_qsum(S, C, red[slot]);
      slot ^= 1;
      if (A.M > 0 && sample_ctr == 0) {
        if (threadIdx.x == 0 && A.r_out) {
          const double Sd = sc.x, Cd = sc.y;
          A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
        }
        ++sample_idx;
      }
      if (A.M > 0 && ++sample_ctr == A.M) sample_ctr = 0;
      float g1[OPT], sn2[OPT], cs2[OPT];
      int S2 = 0, C2 = 0;
      uint32_t tp[OPT];
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        g1[k] = cs[k] * sc.x - sn[k] * sc.y;
        const float d1 = fmaf(A.sc, z[k][s], fmaf(A.kc, g1[k], wdt[k]));
        tp[k] = th[k] + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
      }
      sincos_turns_n<OPT>(tp, sn2, cs2);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn2[k] = cs2[k] = 0.0f;
        S2 += quant(sn2[k]);
        C2 += quant(cs2[k]);
      }
      sc = block_qsum(S2, C2, red[slot]);
      slot ^= 1;
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const float g2 = cs2[k] * sc.x - sn2[k] * sc.y;
        const float d = fmaf(A.sc, z[k][s], fmaf(A.kh, g1[k] + g2, wdt[k]));
        th[k] += (uint32_t)__float2int_rn(d * 4294967296.0f);
      }
    }
    n = (g + 1) << 2;
  }
  // Final sample at n_end.
  if (A.M > 0) {
    int S = 0, C = 0;
#pragma unroll
    for (int k = 0; k < OPT; ++k) {
      float sn, cs;
      sincos_turns(th[k], sn, cs);
      if (valid[k]) {
        S += quant(sn);
        C += quant(cs);
      }
    }
    const float2 sc = block_qsum(S, C, red[slot]);
    if (threadIdx.x == 0 && A.r_out) {
      const double Sd = sc.x, Cd = sc.y;
      A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
    }
  }
  (void)invN;
#pragma unroll
  for (int k = 0; k < OPT; ++k) {
    const int64_t i = threadIdx.x + (int64_t)k * blockDim.x;
    if (valid[k]) A.theta_out[base + i] = th[k];
  }
}

// Mean field with one replica spread over a thread-block cluster of CS CTAs
// (CS from the launch): each CTA holds N / CS oscillators in registers.  Per
// stage every warp reduces its (S, C) with shuffles and stores the pair into
// its slot of every CTA of the cluster (distributed shared memory); one
// cluster barrier later each warp of each CTA sums the CS x warps slots in
// the same fixed order, so all CTAs of a replica use identical sums.  Slots
// are double-buffered across stages, so one barrier per stage suffices.
template <int OPT>
__global__ void __launch_bounds__(512, 1) kur_meanfield_cluster_kernel(const KurArgs A) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int2 slots[2][32];  // [buffer][cluster rank * warps + warp]
  const int cs = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslots = cs * nwarps;  // <= 32, checked by the host
  const int rep = blockIdx.x / cs;
  const int64_t N = A.N;
  const int64_t chunk = (N + cs - 1) / cs;
  const int64_t i0 = (int64_t)crank * chunk;
  const int64_t base = (int64_t)rep * N;
  const uint2 key = seed_to_key(A.seed);
  uint32_t th[OPT];
  float wdt[OPT];
  bool valid[OPT];
  uint32_t oid[OPT];
#pragma unroll
  for (int k = 0; k < OPT; ++k) {
    const int64_t li = threadIdx.x + (int64_t)k * blockDim.x;
    const int64_t i = i0 + li;
    valid[k] = li < chunk && i < N;
    oid[k] = (uint32_t)i;
    th[k] = valid[k] ? A.theta_in[base + i] : 0u;
    wdt[k] = valid[k] ? A.omega[base + i] * A.wscale : 0.0f;
  }
  int buf = 0;
  int64_t sample_ctr = 0, sample_idx = 0;
  // cluster-wide (S, C)
  auto cluster_sum = [&](int S, int C) -> float2 {
    const int2 part = warp_qsum(S, C);
    if (lane < cs) {
      int2 *dst = cluster.map_shared_rank(&slots[buf][crank * nwarps + warp], lane);
      *dst = part;
    }
    cluster.sync();
    const int2 v = lane < nslots ? slots[buf][lane] : make_int2(0, 0);
    buf ^= 1;
    return unquant(warp_qsum(v.x, v.y));
  };
  for (int64_t n = A.n_begin; n < A.n_end;) {
    const int64_t g = n >> 2;
    float z[OPT][4];
#pragma unroll
    for (int k = 0; k < OPT; ++k) gauss4((uint32_t)g, oid[k], (uint32_t)rep, kTagKuramoto, key, z[k]);
    const int s0 = (int)(n & 3);
    const int64_t rem = A.n_end - (g << 2);
    const int s1 = rem < 4 ? (int)rem : 4;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s < s0 || s >= s1) continue;
      float sn[OPT], cs_[OPT];
      int S = 0, C = 0;
      sincos_turns_n<OPT>(th, sn, cs_);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn[k] = cs_[k] = 0.0f;
        S += quant(sn[k]);
        C += quant(cs_[k]);
      }
      float2 sc = cluster_sum(S, C);
      if (A.M > 0 && sample_ctr == 0) {
        if (threadIdx.x == 0 && crank == 0 && A.r_out) {
          const double Sd = sc.x, Cd = sc.y;
          A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
        }
        ++sample_idx;
      }
      if (A.M > 0 && ++sample_ctr == A.M) sample_ctr = 0;
      float g1[OPT], sn2[OPT], cs2[OPT];
      int S2 = 0, C2 = 0;
      uint32_t tp[OPT];
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        g1[k] = cs_[k] * sc.x - sn[k] * sc.y;
        const float d1 = fmaf(A.sc, z[k][s], fmaf(A.kc, g1[k], wdt[k]));
        tp[k] = th[k] + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
      }
      sincos_turns_n<OPT>(tp, sn2, cs2);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn2[k] = cs2[k] = 0.0f;
        S2 += quant(sn2[k]);
        C2 += quant(cs2[k]);
      }
      sc = cluster_sum(S2, C2);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const float g2 = cs2[k] * sc.x - sn2[k] * sc.y;
        const float d = fmaf(A.sc, z[k][s], fmaf(A.kh, g1[k] + g2, wdt[k]));
        th[k] += (uint32_t)__float2int_rn(d * 4294967296.0f);
      }
    }
    n = (g + 1) << 2;
  }
  if (A.M > 0) {
    int S = 0, C = 0;
#pragma unroll
    for (int k = 0; k < OPT; ++k) {
      float sn, c;
      sincos_turns(th[k], sn, c);
      if (valid[k]) {
        S += quant(sn);
        C += quant(c);
      }
    }
    const float2 sc = cluster_sum(S, C);
    if (threadIdx.x == 0 && crank == 0 && A.r_out) {
      const double Sd = sc.x, Cd = sc.y;
      A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
    }
  }
#pragma unroll
  for (int k = 0; k < OPT; ++k)
    if (valid[k]) A.theta_out[base + oid[k]] = th[k];
  cluster.sync();  // no CTA leaves while others may still read its exchange slots
}

// ---- cluster exchange by asynchronous remote stores ----------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait (at most limit_ns) for the phase `parity` of an mbarrier; false on
// expiry.  try_wait may suspend the thread for a while before it answers
// (longer than a short limit: the hardware takes the suspend-time hint as a
// hint only), so limits under a millisecond poll with the non-blocking
// test_wait instead.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = now_ns();
  const bool poll = limit_ns < 1000000ull;
  for (;;) {
    uint32_t done;
    if (poll)
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n\t.reg .pred p;\n\t"
          "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(bar), "r"(parity)
          : "memory");
    if (done) return true;
    if (now_ns() - t0 > limit_ns) return false;
  }
}

// The cluster mean field with the exchange done by st.async: every warp
// sends its (S, C) pair into its slot of every CTA of the cluster with an
// asynchronous remote store that completes on the receiving CTA's mbarrier
// (transaction bytes), and each CTA waits on its own mbarrier for the
// cs x warps pairs of the stage instead of a cluster-wide barrier (whose
// release/acquire fence is what the plain cluster kernel waits on).  Two
// slot buffers and two mbarriers alternate by stage: a CTA can only send
// stage s + 2 after receiving everyone's stage s + 1 pairs, each sent after
// its sender had read the stage s slots, so a buffer is never overwritten
// while it is read, and the receiver has re-armed the buffer's mbarrier
// (after its own stage s wait, before its stage s + 1 sends) before any
// stage s + 2 store can arrive.  Waits are bounded (A.wait_ns, one second by
// default): on expiry the kernel records
// kErrTimeout, leaves the step loop (warp-uniformly) and meets the others at
// the final cluster barrier.
template <int OPT>
__global__ void __launch_bounds__(512, 1) kur_meanfield_async_kernel(const KurArgs A) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ int2 slots[2][32];
  __shared__ __align__(8) uint64_t mbar[2];
  const int cs = (int)cluster.num_blocks();
  const int crank = (int)cluster.block_rank();
  const int nwarps = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nslots = cs * nwarps;  // <= 32, checked by the host
  const uint32_t bytes = (uint32_t)nslots * 8u;
  if (threadIdx.x == 0) {
    // each phase is armed (arrival + expected bytes) before any store of it can
    // arrive: stages 0 and 1 here, stage s + 2 right after stage s completes
    // (no sender reaches stage s + 2 before this CTA has sent stage s + 1)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(bytes)
                 : "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(bytes)
                 : "memory");
  }
  cluster.sync();  // every CTA's barriers exist and are armed before the first remote store
  const int rep = blockIdx.x / cs;
  const int64_t N = A.N;
  const int64_t chunk = (N + cs - 1) / cs;
  const int64_t i0 = (int64_t)crank * chunk;
  const int64_t base = (int64_t)rep * N;
  const uint2 key = seed_to_key(A.seed);
  uint32_t th[OPT];
  float wdt[OPT];
  bool valid[OPT];
  uint32_t oid[OPT];
#pragma unroll
  for (int k = 0; k < OPT; ++k) {
    const int64_t li = threadIdx.x + (int64_t)k * blockDim.x;
    const int64_t i = i0 + li;
    valid[k] = li < chunk && i < N;
    oid[k] = (uint32_t)i;
    th[k] = valid[k] ? A.theta_in[base + i] : 0u;
    wdt[k] = valid[k] ? A.omega[base + i] * A.wscale : 0.0f;
  }
  // remote addresses of this warp's slot and of the mbarriers, in CTA `lane`
  const uint32_t my_slot0 = smem_u32(&slots[0][crank * nwarps + warp]);
  const uint32_t my_slot1 = smem_u32(&slots[1][crank * nwarps + warp]);
  const uint32_t rslot0 = lane < cs ? cluster_map(my_slot0, (uint32_t)lane) : 0u;
  const uint32_t rslot1 = lane < cs ? cluster_map(my_slot1, (uint32_t)lane) : 0u;
  const uint32_t rbar0 = lane < cs ? cluster_map(smem_u32(&mbar[0]), (uint32_t)lane) : 0u;
  const uint32_t rbar1 = lane < cs ? cluster_map(smem_u32(&mbar[1]), (uint32_t)lane) : 0u;
  uint32_t stage = 0;
  bool failed = false;  // warp-uniform
  auto cluster_sum = [&](int S, int C) -> float2 {
    const int2 part = warp_qsum(S, C);
    const int b = (int)(stage & 1u);
    const uint32_t parity = (stage >> 1) & 1u;
    const uint32_t bar = smem_u32(&mbar[b]);
    if (lane < cs)
      asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.s32 [%0], {%1, %2}, [%3];" ::"r"(
                       b ? rslot1 : rslot0),
                   "r"(part.x), "r"(part.y), "r"(b ? rbar1 : rbar0)
                   : "memory");
    const bool ok = mbar_wait_bounded(bar, parity, A.wait_ns);
    if (__any_sync(0xffffffffu, !ok)) {
      failed = true;
      if (lane == 0) atomicOr(A.err, kErrTimeout);
    }
    if (threadIdx.x == 0 && ok)  // arm this buffer's next phase (stage + 2)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    const int2 v = lane < nslots ? slots[b][lane] : make_int2(0, 0);
    ++stage;
    return unquant(warp_qsum(v.x, v.y));
  };
  int64_t sample_ctr = 0, sample_idx = 0;
  for (int64_t n = A.n_begin; n < A.n_end && !failed;) {
    const int64_t g = n >> 2;
    float z[OPT][4];
#pragma unroll
    for (int k = 0; k < OPT; ++k) gauss4((uint32_t)g, oid[k], (uint32_t)rep, kTagKuramoto, key, z[k]);
    const int s0 = (int)(n & 3);
    const int64_t rem = A.n_end - (g << 2);
    const int s1 = rem < 4 ? (int)rem : 4;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (s < s0 || s >= s1 || failed) continue;
      float sn[OPT], cs_[OPT];
      int S = 0, C = 0;
      sincos_turns_n<OPT>(th, sn, cs_);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn[k] = cs_[k] = 0.0f;
        S += quant(sn[k]);
        C += quant(cs_[k]);
      }
      float2 sc = cluster_sum(S, C);
      if (A.M > 0 && sample_ctr == 0) {
        if (threadIdx.x == 0 && crank == 0 && A.r_out) {
          const double Sd = sc.x, Cd = sc.y;
          A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
        }
        ++sample_idx;
      }
      if (A.M > 0 && ++sample_ctr == A.M) sample_ctr = 0;
      float g1[OPT], sn2[OPT], cs2[OPT];
      int S2 = 0, C2 = 0;
      uint32_t tp[OPT];
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        g1[k] = cs_[k] * sc.x - sn[k] * sc.y;
        const float d1 = fmaf(A.sc, z[k][s], fmaf(A.kc, g1[k], wdt[k]));
        tp[k] = th[k] + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
      }
      sincos_turns_n<OPT>(tp, sn2, cs2);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        if (!valid[k]) sn2[k] = cs2[k] = 0.0f;
        S2 += quant(sn2[k]);
        C2 += quant(cs2[k]);
      }
      sc = cluster_sum(S2, C2);
#pragma unroll
      for (int k = 0; k < OPT; ++k) {
        const float g2 = cs2[k] * sc.x - sn2[k] * sc.y;
        const float d = fmaf(A.sc, z[k][s], fmaf(A.kh, g1[k] + g2, wdt[k]));
        th[k] += (uint32_t)__float2int_rn(d * 4294967296.0f);
      }
    }
    n = (g + 1) << 2;
  }
  if (A.M > 0 && !failed) {
    int S = 0, C = 0;
#pragma unroll
    for (int k = 0; k < OPT; ++k) {
      float sn, c;
      sincos_turns(th[k], sn, c);
      if (valid[k]) {
        S += quant(sn);
        C += quant(c);
      }
    }
    const float2 sc = cluster_sum(S, C);
    if (threadIdx.x == 0 && crank == 0 && A.r_out) {
      const double Sd = sc.x, Cd = sc.y;
      A.r_out[sample_idx * A.R + rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
    }
  }
#pragma unroll
  for (int k = 0; k < OPT; ++k)
    if (valid[k]) A.theta_out[base + oid[k]] = th[k];
  cluster.sync();  // no CTA leaves while remote stores into it may be in flight
}

// ---- mean field over the whole grid ------------------------------------

constexpr int kMfgThreads = 256;
constexpr int kMfgIlp = 4;  // oscillators per thread per iteration (loads issued together)

struct MfgArgs {
  uint32_t *theta;    // [R][N] theta_n; the corrector overwrites it with theta_{n+1}
  uint32_t *theta_t;  // [R][N] predictor phases theta~_n
  float *y;           // [R][N] first-stage part of the step: wdt + kh g1 + sc psi
  float *psi;         // [3][R][N] Gaussians of steps 4g+1..4g+3 of the current Philox block
  const float *omega;
  float2 *partials;   // [R][gridDim.x] per-block sums
  double *tot;        // [R][4]: (S, C) of theta_n, then (S, C) of theta~_n
  uint32_t *count;    // [R] blocks finished in this launch (the last one resets it)
  double *r_out;      // [rows][R]
  int64_t N, R;
  int64_t n;           // step index (noise counter)
  int64_t sample_row;  // r row written from this launch's totals, -1 = none
  float wscale, kc, kh, sc;
  PhiloxKeys keys;
};

// MODE 2: sums of (sin, cos) of theta_n.  MODE 0 and 3 (predictor): g1 from the
// totals of theta_n, theta~ = theta + d1, sums over theta~.  MODE 1
// (corrector): g2 from the totals of theta~, theta_{n+1} = theta + y + kh g2,
// sums over theta_{n+1} (the next step's first-stage sums).  The Gaussian of
// step n is element n mod 4 of the Philox block n / 4 of the oscillator (as
// in the other forms): the predictor draws the block at its first step, or
// at the first step of a run (MODE 3), and keeps the later elements in `psi`
// for the next three steps (MODE 0 reads them).  Each thread
// strides over the replica; the block's FP32 sums go to `partials`, and the
// block that finishes last adds all partials of the replica in block order
// in FP64, so the totals do not depend on which block that is.
template <int MODE>
__global__ void __launch_bounds__(kMfgThreads, MODE == 3 ? 4 : (MODE == 2 ? 8 : 5)) kur_mfg_kernel(const MfgArgs A) {
  constexpr bool kPred = MODE == 0 || MODE == 3;
  constexpr bool kGen = MODE == 3;
  __shared__ float2 red[32];
  __shared__ double2 red64[32];
  __shared__ bool is_last;
  const int rep = blockIdx.y;
  const int64_t N = A.N;
  const int64_t NR = N * A.R;
  const int64_t base = (int64_t)rep * N;
  double *tot = A.tot + 4 * rep;
  float S = 0.0f, C = 0.0f;
  if (kPred) {
    S = (float)tot[0];
    C = (float)tot[1];
  } else if (MODE == 1) {
    S = (float)tot[2];
    C = (float)tot[3];
  }
  const int j = (int)(A.n & 3);
  float ps = 0.0f, pc = 0.0f;
  // per-replica base pointers, 32-bit oscillator indices (N < 2^31, so
  // i0 + stride < 2^32 never wraps)
  const uint32_t Nu = (uint32_t)N;
  uint32_t *th_r = A.theta + base;
  uint32_t *tt_r = A.theta_t + base;
  float *y_r = A.y + base;
  const float *om_r = A.omega + base;
  const float *psi_in = (kPred && !kGen && j > 0) ? A.psi + (int64_t)(j - 1) * NR + base : nullptr;
  float *psi_out = A.psi + base;  // plane k - 1 at + (k - 1) NR
  const uint32_t stride = gridDim.x * (uint32_t)(kMfgThreads * kMfgIlp);
  for (uint32_t i0 = blockIdx.x * (uint32_t)(kMfgThreads * kMfgIlp) + threadIdx.x; i0 < Nu; i0 += stride) {
    uint32_t t0[kMfgIlp], tt[kMfgIlp];
    float a1[kMfgIlp], a2[kMfgIlp];
    bool ok[kMfgIlp];
#pragma unroll
    for (int u = 0; u < kMfgIlp; ++u) {
      const uint32_t i = i0 + u * kMfgThreads;
      ok[u] = i < Nu;
      const uint32_t ii = ok[u] ? i : 0u;
      t0[u] = th_r[ii];
      if (kPred) {
        a1[u] = om_r[ii];
        a2[u] = kGen ? 0.0f : psi_in[ii];
      } else if (MODE == 1) {
        tt[u] = tt_r[ii];
        a1[u] = y_r[ii];
      }
    }
    // oscillators u and u + 1 together: their sin/cos polynomials on packed
    // FP32 pairs (sincos_turns2), the rest per oscillator
    static_assert(kMfgIlp % 2 == 0, "oscillators are taken in pairs");
#pragma unroll
    for (int u = 0; u < kMfgIlp; u += 2) {
      float2 sn, cs;
      if (MODE == 2) {
        sincos_turns2(t0[u], t0[u + 1], sn, cs);
      } else if (kPred) {
        float2 s0, c0;
        sincos_turns2(t0[u], t0[u + 1], s0, c0);
        uint32_t tp[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int v = u + e;
          const uint32_t i = i0 + v * kMfgThreads;
          const float g1 = (e ? c0.y : c0.x) * S - (e ? s0.y : s0.x) * C;
          float psi = a2[v];
          if (kGen) {
            float z[4];
            gauss4((uint32_t)(A.n >> 2), i, (uint32_t)rep, kTagKuramoto, A.keys, z);
            psi = pick4(z, j);
            if (ok[v]) {
#pragma unroll
              for (int k = 1; k < 4; ++k)
                if (k > j) psi_out[(int64_t)(k - 1) * NR + i] = z[k];
            }
          }
          const float wdt = a1[v] * A.wscale;
          const float d1 = fmaf(A.sc, psi, fmaf(A.kc, g1, wdt));
          tp[e] = t0[v] + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
          if (ok[v]) {
            tt_r[i] = tp[e];
            y_r[i] = fmaf(A.sc, psi, fmaf(A.kh, g1, wdt));
          }
        }
        sincos_turns2(tp[0], tp[1], sn, cs);
      } else {
        float2 s2, c2;
        sincos_turns2(tt[u], tt[u + 1], s2, c2);
        uint32_t t1[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int v = u + e;
          const uint32_t i = i0 + v * kMfgThreads;
          const float g2 = (e ? c2.y : c2.x) * S - (e ? s2.y : s2.x) * C;
          t1[e] = t0[v] + (uint32_t)__float2int_rn(fmaf(A.kh, g2, a1[v]) * 4294967296.0f);
          if (ok[v]) th_r[i] = t1[e];
        }
        sincos_turns2(t1[0], t1[1], sn, cs);
      }
      if (ok[u]) {
        ps += sn.x;
        pc += cs.x;
      }
      if (ok[u + 1]) {
        ps += sn.y;
        pc += cs.y;
      }
    }
  }
  const float2 b = block_sum2(ps, pc, red);
  if (threadIdx.x == 0) {
    A.partials[(int64_t)rep * gridDim.x + blockIdx.x] = b;
    __threadfence();
    is_last = atomicAdd(&A.count[rep], 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double s = 0.0, c = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += kMfgThreads) {
    const float2 p = __ldcg(&A.partials[(int64_t)rep * gridDim.x + q]);
    s += p.x;
    c += p.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red64[warp] = make_double2(s, c);
  __syncthreads();
  if (threadIdx.x == 0) {
    double S64 = 0.0, C64 = 0.0;
    for (int w = 0; w < kMfgThreads / 32; ++w) {
      S64 += red64[w].x;
      C64 += red64[w].y;
    }
    if (kPred) {
      tot[2] = S64;
      tot[3] = C64;
    } else {
      tot[0] = S64;
      tot[1] = C64;
      if (A.sample_row >= 0 && A.r_out)
        A.r_out[A.sample_row * A.R + rep] = sqrt(S64 * S64 + C64 * C64) / (double)N;
    }
    A.count[rep] = 0u;
  }
}

// ---- pairwise form (Alg. 3) --------------------------------------------

constexpr int kPairThreads = 128;
constexpr int kPairPerThread = 2;  // receivers per thread: one packed FP32 pair
constexpr int kPairTile = kPairThreads * kPairPerThread;

// acc += sin(phi_j - phi_i) for the thread's two receivers i0, i1 and one
// source j, all three phases as 32-bit fixed-point turns.  The difference is
// taken exactly in integers and wraps to [-1/2, 1/2) turn by itself, so no
// range reduction of a float is needed and no receiver carries the rounding
// of its own phase into every one of its terms.  With x = d 2^-32 turns and
// t = 1/4 - ||x| - 1/4| in [0, 1/4] (sin(pi - y) = sin y folds the outer
// quarters onto the inner ones), sin(2 pi x) = sign(x) sin(2 pi t), and
// sin(2 pi t) = t (S0 + S1 t^2 + ... + S4 t^8) with S0 the FP32 value of 2 pi;
// S1..S4 minimise the largest absolute error on a dense grid of [0, 1/4] (a
// linear program, fitted for this library).  In FP32 the result is within
// 2.2e-7 of sin(2 pi x) (RMS 6e-8, no bias).  The polynomial runs on packed
// FP32 pairs, both receivers per instruction, and the special-function unit
// is not used: its sine's error is systematic enough to move phases by ~1e-5
// over 10^3 steps of a partly synchronised population.
__device__ __forceinline__ void pair_terms2(uint32_t tj, uint32_t ti0, uint32_t ti1, float2 &acc) {
  const float2 x = __fmul2_rn(make_float2((float)(int32_t)(tj - ti0), (float)(int32_t)(tj - ti1)),
                              make_float2(2.3283064365386963e-10f, 2.3283064365386963e-10f));  // 2^-32
  const float2 u = __fadd2_rn(make_float2(fabsf(x.x), fabsf(x.y)), make_float2(-0.25f, -0.25f));
  const float2 t = __fadd2_rn(make_float2(0.25f, 0.25f), make_float2(-fabsf(u.x), -fabsf(u.y)));
  const float2 t2 = __fmul2_rn(t, t);
  float2 p = __ffma2_rn(t2, make_float2(3.903203201e+01f, 3.903203201e+01f),
                        make_float2(-7.653708649e+01f, -7.653708649e+01f));
  p = __ffma2_rn(p, t2, make_float2(8.160352325e+01f, 8.160352325e+01f));
  p = __ffma2_rn(p, t2, make_float2(-4.134174728e+01f, -4.134174728e+01f));
  p = __ffma2_rn(p, t2, make_float2(6.283185482e+00f, 6.283185482e+00f));
  acc = __ffma2_rn(make_float2(copysignf(t.x, x.x), copysignf(t.y, x.y)), p, acc);
}

// One SRK2 stage: receivers i of one replica in this CTA, all sources j
// streamed through shared memory in tiles.  STAGE 0 (predictor) reads the
// phases theta, writes theta~ and the first-stage coupling sum g1; STAGE 1
// (corrector) takes the sums over theta~ and writes the new theta.  STAGE 2
// is PROG2's UpdateRHS: the sums over theta, stored in g1 for the
// AdvanceSystem kernel of the Euler-Maruyama scheme.
template <int STAGE>
__global__ void __launch_bounds__(kPairThreads) kur_pairwise_stage(const KurPairArgs A) {
  __shared__ uint4 src_s[kPairTile / 4];  // source phases (fixed-point turns), four per entry
  const int rep = blockIdx.y;
  const int64_t N = A.N;
  const int64_t base = (int64_t)rep * N;
  const uint32_t *src = STAGE == 1 ? A.theta_t : A.theta;  // corrector: sums over theta~
  uint32_t ti[kPairPerThread];
  float acc[kPairPerThread];
  int64_t idx[kPairPerThread];
#pragma unroll
  for (int k = 0; k < kPairPerThread; ++k) {
    idx[k] = (int64_t)blockIdx.x * kPairTile + threadIdx.x + k * kPairThreads;
    ti[k] = idx[k] < N ? src[base + idx[k]] : 0u;
    acc[k] = 0.0f;
  }
  static_assert(kPairPerThread == 2, "the receivers of a thread form one packed pair");
  uint32_t *src_w = reinterpret_cast<uint32_t *>(src_s);
  float2 acc2 = make_float2(0.0f, 0.0f);
  for (int64_t j0 = 0; j0 < N; j0 += kPairTile) {
    const int cnt = (N - j0) < kPairTile ? (int)(N - j0) : kPairTile;
#pragma unroll
    for (int k = 0; k < kPairPerThread; ++k) {
      const int jj = threadIdx.x + k * kPairThreads;
      if (jj < cnt) src_w[jj] = src[base + j0 + jj];
    }
    __syncthreads();
    if (cnt == kPairTile) {
#pragma unroll 2
      for (int q = 0; q < kPairTile / 4; ++q) {
        const uint4 t4 = src_s[q];
        pair_terms2(t4.x, ti[0], ti[1], acc2);
        pair_terms2(t4.y, ti[0], ti[1], acc2);
        pair_terms2(t4.z, ti[0], ti[1], acc2);
        pair_terms2(t4.w, ti[0], ti[1], acc2);
      }
    } else {
      for (int jj = 0; jj < cnt; ++jj) pair_terms2(src_w[jj], ti[0], ti[1], acc2);
    }
    __syncthreads();
  }
  acc[0] = acc2.x;
  acc[1] = acc2.y;
  if (STAGE == 2) {
#pragma unroll
    for (int k = 0; k < kPairPerThread; ++k)
      if (idx[k] < N) A.g1[base + idx[k]] = acc[k];
    return;
  }
  const uint2 key = seed_to_key(A.seed);
  const int64_t n = A.n;
#pragma unroll
  for (int k = 0; k < kPairPerThread; ++k) {
    if (idx[k] >= N) continue;
    const int64_t gi = base + idx[k];
    float z[4];
    gauss4((uint32_t)(n >> 2), (uint32_t)idx[k], (uint32_t)rep, kTagKuramoto, key, z);
    const float psi = pick4(z, (int)(n & 3));
    const float wdt = A.omega[gi] * A.wscale;
    if (STAGE == 0) {
      const float d1 = fmaf(A.sc, psi, fmaf(A.kc, acc[k], wdt));
      A.theta_t[gi] = A.theta[gi] + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
      A.g1[gi] = acc[k];
    } else {
      const float d = fmaf(A.sc, psi, fmaf(A.kh, A.g1[gi] + acc[k], wdt));
      A.theta[gi] += (uint32_t)__float2int_rn(d * 4294967296.0f);
    }
  }
}

// PROG2's AdvanceSystem with Euler-Maruyama: theta += wdt + kc g + sc psi
// for every oscillator of every replica, g the stored coupling sums.
__global__ void kur_advance_euler_kernel(const KurPairArgs A, int64_t R) {
  const uint2 key = seed_to_key(A.seed);
  const int64_t NR = A.N * R;
  for (int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; gi < NR;
       gi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rep = gi / A.N, i = gi - rep * A.N;
    float z[4];
    gauss4((uint32_t)(A.n >> 2), (uint32_t)i, (uint32_t)rep, kTagKuramoto, key, z);
    const float d = fmaf(A.sc, pick4(z, (int)(A.n & 3)), fmaf(A.kc, A.g1[gi], A.omega[gi] * A.wscale));
    A.theta[gi] += (uint32_t)__float2int_rn(d * 4294967296.0f);
  }
}

// r(t) of every replica from fixed-point phases (one CTA per replica).
__global__ void kur_order_kernel(const uint32_t *theta, int64_t N, int64_t R, double *r_out) {
  __shared__ float2 red[32];
  const int rep = blockIdx.x;
  float S = 0.0f, C = 0.0f;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    float sn, cs;
    sincos_turns(theta[(int64_t)rep * N + i], sn, cs);
    S += sn;
    C += cs;
  }
  const float2 sc = block_sum2(S, C, red);
  if (threadIdx.x == 0) {
    const double Sd = sc.x, Cd = sc.y;
    r_out[rep] = sqrt(Sd * Sd + Cd * Cd) / (double)N;
  }
}

// Radians (any range) <-> fixed-point turns.
__global__ void kur_to_fixed(const float *phi, uint32_t *theta, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double t = (double)phi[i] * 0.15915494309189533577;  // 1 / (2 pi)
    t -= floor(t);
    theta[i] = (uint32_t)(uint64_t)llrint(t * 4294967296.0);
  }
}

__global__ void kur_from_fixed(const uint32_t *theta, float *phi, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    phi[i] = (float)((double)theta[i] * 2.3283064365386963e-10 * 6.28318530717958647692);
}

// Observables: mean, variance and standard error of r over replicas for
// each sample row (one warp per row, fixed summation order).
__global__ void kur_obs_kernel(const double *r, int64_t rows, int64_t R, int64_t n_begin, int64_t n_end,
                               int M, double dt, sde_obs_row *obs) {
  const int64_t row = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  double s = 0.0;
  for (int64_t q = lane; q < R; q += 32) s += r[row * R + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const double mean = s / (double)R;
  double m2 = 0.0;
  for (int64_t q = lane; q < R; q += 32) {
    const double d = r[row * R + q] - mean;
    m2 += d * d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, o);
  if (lane == 0) {
    sde_obs_row o;
    o.mean = mean;
    o.count = (double)R;
    o.var = R > 1 ? m2 / (double)(R - 1) : 0.0;
    o.se = sqrt(o.var / (double)R);
    const int64_t n = row == rows - 1 ? n_end : n_begin + row * (int64_t)M;
    o.t = (double)n * dt;
    obs[row] = o;
  }
}

// Direct coupling sums for the uniform models: out[r][i] = (K/N) sum_j
// sin(x_j - x_i), accurate sinpif per pair (inspection path, not the
// integrator).
__global__ void kur_coupling_uniform_kernel(const uint32_t *theta, float *out, int64_t N, float KoverN) {
  __shared__ float src_s[256];
  const int rep = blockIdx.y;
  const int64_t base = (int64_t)rep * N;
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const float ti = i < N ? (float)(int32_t)theta[base + i] * 2.3283064365386963e-10f : 0.0f;
  float acc = 0.0f;
  for (int64_t j0 = 0; j0 < N; j0 += 256) {
    const int cnt = (N - j0) < 256 ? (int)(N - j0) : 256;
    if (threadIdx.x < cnt) src_s[threadIdx.x] = (float)(int32_t)theta[base + j0 + threadIdx.x] * 2.3283064365386963e-10f;
    __syncthreads();
    for (int jj = 0; jj < cnt; ++jj) {
      float d = src_s[jj] - ti;
      d -= rintf(d);
      acc += sinpif(2.0f * d);
    }
    __syncthreads();
  }
  if (i < N) out[base + i] = KoverN * acc;
}

template <int OPT>
void *mf_kernel_ptr() {
  return (void *)kur_meanfield_kernel<OPT>;
}

template <int OPT>
cudaError_t launch_mf_cluster(const KurArgs &a, int block, int cs, bool async, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.R * cs));
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (async) return cudaLaunchKernelEx(&cfg, kur_meanfield_async_kernel<OPT>, a);
  return cudaLaunchKernelEx(&cfg, kur_meanfield_cluster_kernel<OPT>, a);
}

// cs > 1: one replica per cluster of cs CTAs (opt oscillators per thread of
// each CTA); cs == 1: one CTA per replica.
cudaError_t launch_meanfield(const KurArgs &a, int block, int opt, int cs, bool async, cudaStream_t s) {
  if (cs > 1) {
    switch (opt) {
      case 1: return launch_mf_cluster<1>(a, block, cs, async, s);
      case 2: return launch_mf_cluster<2>(a, block, cs, async, s);
      case 4: return launch_mf_cluster<4>(a, block, cs, async, s);
      case 8: return launch_mf_cluster<8>(a, block, cs, async, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (opt) {
    case 1: kur_meanfield_kernel<1><<<(unsigned)a.R, block, 0, s>>>(a); break;
    case 2: kur_meanfield_kernel<2><<<(unsigned)a.R, block, 0, s>>>(a); break;
    case 4: kur_meanfield_kernel<4><<<(unsigned)a.R, block, 0, s>>>(a); break;
    case 8: kur_meanfield_kernel<8><<<(unsigned)a.R, block, 0, s>>>(a); break;
    case 16: kur_meanfield_kernel<16><<<(unsigned)a.R, block, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Blocks per replica of the grid-wide mean field: enough oscillators per
// thread to amortise the reduction, about eight blocks per SM in total.
// One full wave of each kernel (resident blocks per SM from the occupancy
// calculator x SMs, shared among the replicas), at most one block per
// kMfgThreads x kMfgIlp oscillators.
void mfg_grid_for(int64_t N, int64_t R, int sm_count, int grid[4]) {
  const void *fn[4] = {(const void *)kur_mfg_kernel<0>, (const void *)kur_mfg_kernel<1>,
                       (const void *)kur_mfg_kernel<2>, (const void *)kur_mfg_kernel<3>};
  const int64_t need = (N + kMfgThreads * kMfgIlp - 1) / (kMfgThreads * kMfgIlp);
  for (int m = 0; m < 4; ++m) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn[m], kMfgThreads, 0) != cudaSuccess)
      per_sm = 4;
    const int64_t fill = std::max<int64_t>(1, ((int64_t)std::max(1, per_sm) * sm_count + R - 1) / R);
    grid[m] = (int)std::max<int64_t>(1, std::min<int64_t>(need, fill));
  }
}

cudaError_t launch_mfg(const MfgArgs &a, int mode, int blocks, cudaStream_t s) {
  const dim3 grid((unsigned)blocks, (unsigned)a.R);
  switch (mode) {
    case 0: kur_mfg_kernel<0><<<grid, kMfgThreads, 0, s>>>(a); break;
    case 1: kur_mfg_kernel<1><<<grid, kMfgThreads, 0, s>>>(a); break;
    case 3: kur_mfg_kernel<3><<<grid, kMfgThreads, 0, s>>>(a); break;
    default: kur_mfg_kernel<2><<<grid, kMfgThreads, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

int pow2_at_least(int64_t x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------

namespace {

struct MfShape {
  int cs, block, opt;
  bool async;  // cluster exchange by st.async + mbarrier instead of a cluster barrier
};

// Candidate shapes for the mean-field kernel: one CTA per replica, or a
// cluster of 2, 4 or 8 CTAs per replica (distributed shared memory
// reductions; more, smaller CTAs let co-resident replicas overlap each
// other's barrier latency).
std::vector<MfShape> meanfield_candidates(int64_t N) {
  std::vector<MfShape> out;
  for (int cs : {1, 2, 4, 8}) {
    const int64_t chunk = (N + cs - 1) / cs;
    for (int block : {128, 256, 512, 1024}) {
      if (block == 128 && cs < 8) continue;
      if (cs > 1 && cs * (block / 32) > 32) continue;  // one exchange slot per warp of the cluster
      if (block > ((chunk + 31) / 32) * 32 && block > 256) continue;  // mostly idle threads
      const int opt = pow2_at_least((chunk + block - 1) / block);
      const int max_opt = cs > 1 ? 8 : 16;
      const int max_block = cs > 1 ? 512 : (opt <= 2 ? 1024 : 512);
      if (opt > max_opt || block > max_block) continue;
      out.push_back({cs, block, opt, false});
      if (cs > 1) out.push_back({cs, block, opt, true});
    }
  }
  return out;
}

}  // namespace

MfgArgs mfg_args(KuramotoCtx *k, const float *omega, double *rbuf) {
  const double inv2pi = 0.15915494309189533577;
  MfgArgs a{};
  a.theta = k->theta;
  a.theta_t = k->theta_t;
  a.y = k->g1;
  a.psi = k->psi4;
  a.omega = omega;
  a.partials = k->mfg_partials;
  a.tot = k->mfg_tot;
  a.count = k->mfg_count;
  a.r_out = rbuf;
  a.N = k->N;
  a.R = k->R;
  a.wscale = (float)(k->dt * inv2pi);
  a.kc = (float)(k->K / (double)k->N * k->dt * inv2pi);
  a.kh = (float)(0.5 * k->K / (double)k->N * k->dt * inv2pi);
  a.sc = (float)(sqrt(2.0 * k->D * k->dt) * inv2pi);
  a.keys = philox_round_keys(k->seed);
  return a;
}

// Steps [n_begin, n_end) of the grid-wide mean field: the sums of theta at
// n_begin, then predictor and corrector launches per step.  r(t) rows as in
// the single-CTA form: every M steps from n_begin, plus n_end as the last row.
sde_status run_meanfield_grid(KuramotoCtx *k, int64_t n_begin, int64_t n_end, const float *omega,
                              double *rbuf, int64_t n_rows, cudaStream_t s) {
  MfgArgs a = mfg_args(k, omega, rbuf);
  const int *grid = k->mfg_grid;
  a.n = n_begin;
  a.sample_row = n_rows > 0 ? 0 : -1;
  SDE_CUDA_TRY(launch_mfg(a, 2, grid[2], s));
  for (int64_t n = n_begin; n < n_end; ++n) {
    a.n = n;
    const int pred = (n == n_begin || (n & 3) == 0) ? 3 : 0;
    a.sample_row = -1;
    SDE_CUDA_TRY(ktime_begin(k, s));
    SDE_CUDA_TRY(launch_mfg(a, pred, grid[pred], s));
    SDE_CUDA_TRY(ktime_end(k, s));
    const int64_t m = n + 1;
    if (n_rows > 0) {
      if (m == n_end)
        a.sample_row = n_rows - 1;
      else if ((m - n_begin) % k->M == 0)
        a.sample_row = (m - n_begin) / k->M;
    }
    SDE_CUDA_TRY(ktime_begin(k, s));
    SDE_CUDA_TRY(launch_mfg(a, 1, grid[1], s));
    SDE_CUDA_TRY(ktime_end(k, s));
  }
  return SDE_OK;
}

// Time a short run of every candidate shape on scratch phases and keep the
// fastest.
sde_status meanfield_autotune(KuramotoCtx *k, int only_cs, bool with_grid) {
  auto cands = meanfield_candidates(k->N);
  if (k->flags & SDE_FLAG_ASYNC_EXCHANGE) {
    std::vector<MfShape> keep;
    for (const auto &c : cands)
      if (c.async) keep.push_back(c);
    cands.swap(keep);
  } else if (with_grid && only_cs == 0) {
    cands.push_back({0, kMfgThreads, 0, false});
  }
  if (only_cs > 0) {
    std::vector<MfShape> keep;
    for (const auto &c : cands)
      if (c.cs == only_cs) keep.push_back(c);
    cands.swap(keep);
  }
  if (cands.empty()) {
    set_error("invalid argument: no mean-field launch shape holds n_osc = " + std::to_string(k->N));
    return SDE_ERR_INVALID_ARG;
  }
  const size_t NR = (size_t)k->N * (size_t)k->R;
  float *omega = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sde_status st = SDE_OK;
  cudaError_t e;
  if ((e = device_alloc((void **)&omega, NR * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) st = cuda_fail(e, "stream");
  if (st == SDE_OK && (e = cudaEventCreate(&e0)) != cudaSuccess) st = cuda_fail(e, "event");
  if (st == SDE_OK && (e = cudaEventCreate(&e1)) != cudaSuccess) st = cuda_fail(e, "event");
  if (st == SDE_OK) {
    cudaMemsetAsync(omega, 0, NR * 4, s);
    cudaMemsetAsync(k->theta, 0, NR * 4, s);
    KurArgs a{};
    a.theta_in = k->theta;
    a.theta_out = k->theta;
    a.omega = omega;
    a.r_out = nullptr;
    a.N = k->N;
    a.R = k->R;
    a.n_begin = 0;
    a.n_end = 64;
    a.M = 0;
    a.wscale = 1e-3f;
    a.kc = 1e-4f;
    a.kh = 5e-5f;
    a.sc = 1e-3f;
    a.seed = 0;
    a.err = k->err;
    a.wait_ns = k->wait_ns;
    float best = 1e30f;
    for (const MfShape &c : cands) {
      float tmin = 1e30f;
      for (int rep = 0; rep < 3 && st == SDE_OK; ++rep) {
        cudaEventRecord(e0, s);
        if (c.cs == 0) {
          const uint32_t flags = k->flags;
          k->flags &= ~SDE_FLAG_TIME_KERNELS;
          st = run_meanfield_grid(k, a.n_begin, a.n_end, omega, nullptr, 0, s);
          k->flags = flags;
          if (st != SDE_OK) break;
        } else if ((e = launch_meanfield(a, c.block, c.opt, c.cs, c.async, s)) != cudaSuccess) {
          st = cuda_fail(e, "mean-field autotune launch");
          break;
        }
        cudaEventRecord(e1, s);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
          st = cuda_fail(e, "mean-field autotune");
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);
      }
      if (st != SDE_OK) break;
      if (tmin < best) {
        best = tmin;
        k->cs = c.cs;
        k->mf_async = c.async;
        k->block = c.block;
        k->opt = c.opt;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  cudaFree(omega);
  if (st == SDE_OK) cudaMemset(k->err, 0, sizeof(uint32_t));  // scratch runs report nothing
  return st;
}

sde_status kuramoto_validate(const sde_config *cfg) {
  SDE_CHECK_ARG(cfg->n_osc >= 1, "n_osc must be >= 1");
  SDE_CHECK_ARG(cfg->n_replicas >= 1 && cfg->n_replicas <= 65535, "n_replicas must be in [1, 65535]");
  SDE_CHECK_ARG(isfinite(cfg->K) && isfinite(cfg->D) && isfinite(cfg->dt), "K, D, dt must be finite");
  SDE_CHECK_ARG(cfg->D >= 0.0, "D must be >= 0");
  SDE_CHECK_ARG(cfg->dt > 0.0, "dt must be > 0");
  SDE_CHECK_ARG(cfg->sample_every >= 0, "sample_every must be >= 0");
  SDE_CHECK_ARG(cfg->n_osc < (1ll << 31), "n_osc too large");
  if (cfg->flags & SDE_FLAG_EULER) {
    if (cfg->model != SDE_KURAMOTO_PAIRWISE) {
      set_error("unsupported: Euler-Maruyama (SDE_FLAG_EULER) is built for the Josephson and the "
                "pairwise Kuramoto models");
      return SDE_ERR_UNSUPPORTED;
    }
  }
  const bool mf = cfg->model == SDE_KURAMOTO_MEANFIELD;
  if (mf)
    SDE_CHECK_ARG(cfg->schedule == SDE_SCHED_PERSISTENT || cfg->schedule == SDE_SCHED_GRID,
                  "mean-field schedule must be SDE_SCHED_PERSISTENT (choose the form) or SDE_SCHED_GRID");
  else
    SDE_CHECK_ARG(cfg->schedule == SDE_SCHED_PERSISTENT, "schedule must be 0 for this Kuramoto model");
  // Forms of the mean field: a replica per CTA or cluster (n_osc <= 8192), or
  // spread over the whole grid (any n_osc; forced by SDE_SCHED_GRID).
  const bool grid_forced = mf && (cfg->schedule == SDE_SCHED_GRID || cfg->n_osc > 8192);
  if (grid_forced)
    SDE_CHECK_ARG(cfg->cluster_ctas == 0 && cfg->block_threads == 0,
                  "the grid-wide mean field takes cluster_ctas = 0 and block_threads = 0");
  return SDE_OK;
}

sde_status kuramoto_create(const sde_config *cfg, int sm_count, uint32_t *err, KuramotoCtx **out) {
  *out = nullptr;
  const sde_status vs = kuramoto_validate(cfg);
  if (vs != SDE_OK) return vs;
  const bool mf = cfg->model == SDE_KURAMOTO_MEANFIELD;
  const bool grid_forced = mf && (cfg->schedule == SDE_SCHED_GRID || cfg->n_osc > 8192);
  KuramotoCtx *k = new (std::nothrow) KuramotoCtx();
  if (!k) {
    set_error("host allocation failed");
    return SDE_ERR_NO_MEMORY;
  }
  k->model = cfg->model;
  k->N = cfg->n_osc;
  k->R = cfg->n_replicas;
  k->K = cfg->K;
  k->D = cfg->D;
  k->dt = cfg->dt;
  k->M = cfg->sample_every;
  k->seed = cfg->seed;
  k->sm_count = sm_count;
  k->err = err;
  k->flags = cfg->flags;
  const size_t NR = (size_t)k->N * (size_t)k->R;
  sde_status st = SDE_OK;
  cudaError_t e;
  auto alloc = [&](void **p, size_t bytes) {
    if (st != SDE_OK) return;
    if ((e = device_alloc(p, bytes ? bytes : 1)) != cudaSuccess) st = cuda_fail(e, "cudaMalloc");
  };
  alloc((void **)&k->theta, NR * 4);
  // the grid-wide form is a candidate when few replicas leave SMs idle
  const bool grid_possible =
      mf && (grid_forced || (cfg->cluster_ctas == 0 && cfg->block_threads == 0 && cfg->n_replicas * 4 < sm_count));
  if (cfg->model == SDE_KURAMOTO_PAIRWISE || grid_possible) {
    alloc((void **)&k->theta_t, NR * 4);
    alloc((void **)&k->g1, NR * 4);
  }
  if (grid_possible) {
    mfg_grid_for(k->N, k->R, sm_count, k->mfg_grid);
    k->mfg_blocks = *std::max_element(k->mfg_grid, k->mfg_grid + 4);
    alloc((void **)&k->mfg_partials, sizeof(float2) * (size_t)k->mfg_blocks * (size_t)k->R);
    alloc((void **)&k->mfg_tot, sizeof(double) * 4 * (size_t)k->R);
    alloc((void **)&k->mfg_count, sizeof(uint32_t) * (size_t)k->R);
    alloc((void **)&k->psi4, sizeof(float) * 3 * NR);
    if (st == SDE_OK && (e = cudaMemset(k->mfg_count, 0, sizeof(uint32_t) * (size_t)k->R)) != cudaSuccess)
      st = cuda_fail(e, "cudaMemset");
  }
  if (st == SDE_OK && (cfg->model == SDE_KURAMOTO_GENERAL || cfg->model == SDE_KURAMOTO_GENERAL_FP32))
    st = kuramoto_general_alloc(k);
  if (st != SDE_OK) {
    kuramoto_destroy(k);
    return st;
  }
  // Launch shape.
  SDE_CHECK_ARG(cfg->cluster_ctas == 0 || cfg->cluster_ctas == 1 || cfg->cluster_ctas == 2 ||
                    cfg->cluster_ctas == 4 || cfg->cluster_ctas == 8,
                "cluster_ctas must be 0, 1, 2, 4 or 8");
  if (grid_forced) {
    k->cs = 0;
    k->block = kMfgThreads;
  } else if (cfg->model == SDE_KURAMOTO_MEANFIELD && cfg->block_threads == 0) {
    st = meanfield_autotune(k, cfg->cluster_ctas, grid_possible);
    if (st != SDE_OK) {
      kuramoto_destroy(k);
      return st;
    }
  } else if (cfg->model == SDE_KURAMOTO_MEANFIELD && cfg->cluster_ctas > 1) {
    // a fixed cluster shape: cs CTAs of block threads per replica
    const int cs = cfg->cluster_ctas, block = cfg->block_threads;
    const int64_t chunk = (k->N + cs - 1) / cs;
    const int opt = pow2_at_least((chunk + block - 1) / block);
    if (block < 32 || block % 32 != 0 || block > 512 || cs * (block / 32) > 32 || opt > 8) {
      kuramoto_destroy(k);
      set_error("invalid argument: with cluster_ctas > 1, block_threads must be a multiple of 32, at most "
                "512 and at most 32 warps per cluster, with at most 8 oscillators per thread");
      return SDE_ERR_INVALID_ARG;
    }
    k->cs = cs;
    k->block = block;
    k->opt = opt;
    k->mf_async = (cfg->flags & SDE_FLAG_ASYNC_EXCHANGE) != 0;
  } else if (cfg->model == SDE_KURAMOTO_MEANFIELD) {
    int block = cfg->block_threads;
    int opt = pow2_at_least((k->N + block - 1) / block);
    if (block < 32 || block % 32 != 0 || block > (opt <= 2 ? 1024 : 512) || opt > 16) {
      kuramoto_destroy(k);
      set_error("invalid argument: block_threads must be a multiple of 32, at most 1024 for <= 2 "
                "oscillators per thread and 512 above, with at most 16 oscillators per thread");
      return SDE_ERR_INVALID_ARG;
    }
    k->block = block;
    k->opt = opt;
  } else if (cfg->model == SDE_KURAMOTO_PAIRWISE) {
    k->block = kPairThreads;
    k->opt = kPairPerThread;
  }
  *out = k;
  return SDE_OK;
}

void kuramoto_tuning(const KuramotoCtx *k, int32_t *block, int32_t *per_thread, int32_t *cluster) {
  if (block) *block = k->block;
  if (per_thread)
    *per_thread = (k->model == SDE_KURAMOTO_MEANFIELD && k->cs == 0)
                      ? (int32_t)((k->N + (int64_t)k->mfg_grid[0] * kMfgThreads - 1) /
                                  ((int64_t)k->mfg_grid[0] * kMfgThreads))
                      : k->opt;
  if (cluster) *cluster = k->cs;
}

cudaError_t ktime_begin(KuramotoCtx *k, cudaStream_t s) {
  if (!(k->flags & SDE_FLAG_TIME_KERNELS)) return cudaSuccess;
  while ((int64_t)k->kev.size() < 2 * (k->kev_used + 1)) {
    cudaEvent_t e;
    const cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return err;
    k->kev.push_back(e);
  }
  return cudaEventRecord(k->kev[2 * k->kev_used], s);
}

cudaError_t ktime_end(KuramotoCtx *k, cudaStream_t s, int64_t launches) {
  if (!(k->flags & SDE_FLAG_TIME_KERNELS)) return cudaSuccess;
  const cudaError_t err = cudaEventRecord(k->kev[2 * k->kev_used + 1], s);
  ++k->kev_used;
  k->kev_launches += launches;
  return err;
}

bool kuramoto_kernel_stats(KuramotoCtx *k, float *mean_ms, float *total_ms, int64_t *launches) {
  if (k->kev_used == 0) return false;
  if (cudaEventSynchronize(k->kev[2 * k->kev_used - 1]) != cudaSuccess) return false;
  double tot = 0.0;
  for (int64_t i = 0; i < k->kev_used; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, k->kev[2 * i], k->kev[2 * i + 1]) != cudaSuccess) return false;
    tot += ms;
  }
  if (total_ms) *total_ms = (float)tot;
  if (k->kev_launches == 0) return false;
  if (mean_ms) *mean_ms = (float)(tot / (double)k->kev_launches);
  if (launches) *launches = k->kev_launches;
  return true;
}

void kuramoto_set_wait_limit(KuramotoCtx *k, uint64_t ns) {
  if (k) k->wait_ns = ns;
}

void kuramoto_destroy(KuramotoCtx *k) {
  if (!k) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : k->kev) cudaEventDestroy(e);
  cudaFree(k->theta);
  cudaFree(k->theta_t);
  cudaFree(k->g1);
  cudaFree(k->r_scratch);
  cudaFree(k->mfg_partials);
  cudaFree(k->mfg_tot);
  cudaFree(k->mfg_count);
  kuramoto_general_free(k);
  delete k;
}

sde_status kuramoto_run(KuramotoCtx *k, const sde_run_desc *r, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1, sde_obs_row *obs_in, sde_obs_row **obs, int64_t *max_rows,
                        int64_t *rows) {
  SDE_CHECK_ARG(r->phi_in_dev && r->phi_out_dev && r->omega_dev,
                "Kuramoto run needs phi_in, phi_out and omega");
  const int64_t L = r->n_end - r->n_begin;
  const int64_t n_rows = k->M > 0 ? (L + k->M - 1) / k->M + 1 : 0;
  // Observable and sample buffers.
  if (n_rows > *max_rows) {
    cudaFree(obs_in);
    *obs = nullptr;
    *max_rows = 0;
    SDE_CUDA_TRY(device_alloc((void **)obs, sizeof(sde_obs_row) * n_rows));
    *max_rows = n_rows;
  }
  double *rbuf = r->r_out_dev;
  if (!rbuf && n_rows > 0) {
    if (k->r_scratch_rows < n_rows) {
      cudaFree(k->r_scratch);
      k->r_scratch = nullptr;
      k->r_scratch_rows = 0;
      SDE_CUDA_TRY(device_alloc((void **)&k->r_scratch, sizeof(double) * n_rows * k->R));
      k->r_scratch_rows = n_rows;
    }
    rbuf = k->r_scratch;
  }
  const int64_t NR = k->N * k->R;
  const int cvt_grid = (int)std::min<int64_t>((NR + 255) / 256, 4096);
  kur_to_fixed<<<cvt_grid, 256, 0, s>>>(r->phi_in_dev, k->theta, NR);
  SDE_CUDA_TRY(cudaGetLastError());
  const double inv2pi = 0.15915494309189533577;
  k->kev_used = 0;
  k->kev_launches = 0;
  SDE_CUDA_TRY(cudaEventRecord(ev0, s));
  if (k->model == SDE_KURAMOTO_MEANFIELD && k->cs == 0) {
    sde_status st = run_meanfield_grid(k, r->n_begin, r->n_end, r->omega_dev, rbuf, n_rows, s);
    if (st != SDE_OK) return st;
  } else if (k->model == SDE_KURAMOTO_MEANFIELD) {
    KurArgs a{};
    a.theta_in = k->theta;
    a.theta_out = k->theta;
    a.omega = r->omega_dev;
    a.r_out = rbuf;
    a.N = k->N;
    a.R = k->R;
    a.n_begin = r->n_begin;
    a.n_end = r->n_end;
    a.M = k->M;
    a.wscale = (float)(k->dt * inv2pi);
    a.kc = (float)(k->K / (double)k->N * k->dt * inv2pi);
    a.kh = (float)(0.5 * k->K / (double)k->N * k->dt * inv2pi);
    a.sc = (float)(sqrt(2.0 * k->D * k->dt) * inv2pi);
    a.seed = k->seed;
    a.err = k->err;
    a.wait_ns = k->wait_ns;
    SDE_CUDA_TRY(launch_meanfield(a, k->block, k->opt, k->cs, k->mf_async, s));
  } else if (k->model == SDE_KURAMOTO_PAIRWISE) {
    KurPairArgs a{};
    a.theta = k->theta;
    a.theta_t = k->theta_t;
    a.g1 = k->g1;
    a.omega = r->omega_dev;
    a.N = k->N;
    a.wscale = (float)(k->dt * inv2pi);
    a.kc = (float)(k->K / (double)k->N * k->dt * inv2pi);
    a.kh = (float)(0.5 * k->K / (double)k->N * k->dt * inv2pi);
    a.sc = (float)(sqrt(2.0 * k->D * k->dt) * inv2pi);
    a.seed = k->seed;
    const dim3 grid((unsigned)((k->N + kPairTile - 1) / kPairTile), (unsigned)k->R);
    int64_t sample = 0;
    const bool euler = (k->flags & SDE_FLAG_EULER) != 0;
    const int64_t NR = k->N * k->R;
    const unsigned adv_grid = (unsigned)std::min<int64_t>((NR + 255) / 256, (int64_t)k->sm_count * 8);
    for (int64_t n = r->n_begin; n < r->n_end; ++n) {
      if (k->M > 0 && (n - r->n_begin) % k->M == 0) {
        kur_order_kernel<<<(unsigned)k->R, 256, 0, s>>>(k->theta, k->N, k->R, rbuf + sample * k->R);
        ++sample;
      }
      a.n = n;
      if (euler) {
        // PROG2: UpdateRHS, then AdvanceSystem
        SDE_CUDA_TRY(ktime_begin(k, s));
        kur_pairwise_stage<2><<<grid, kPairThreads, 0, s>>>(a);
        SDE_CUDA_TRY(ktime_end(k, s));
        kur_advance_euler_kernel<<<adv_grid, 256, 0, s>>>(a, k->R);
        continue;
      }
      SDE_CUDA_TRY(ktime_begin(k, s));
      kur_pairwise_stage<0><<<grid, kPairThreads, 0, s>>>(a);
      SDE_CUDA_TRY(ktime_end(k, s));
      SDE_CUDA_TRY(ktime_begin(k, s));
      kur_pairwise_stage<1><<<grid, kPairThreads, 0, s>>>(a);
      SDE_CUDA_TRY(ktime_end(k, s));
    }
    SDE_CUDA_TRY(cudaGetLastError());
    if (k->M > 0) kur_order_kernel<<<(unsigned)k->R, 256, 0, s>>>(k->theta, k->N, k->R, rbuf + sample * k->R);
  } else {
    sde_status st = kuramoto_general_run(k, r, s, rbuf);
    if (st != SDE_OK) return st;
  }
  SDE_CUDA_TRY(cudaGetLastError());
  SDE_CUDA_TRY(cudaEventRecord(ev1, s));
  kur_from_fixed<<<cvt_grid, 256, 0, s>>>(k->theta, r->phi_out_dev, NR);
  SDE_CUDA_TRY(cudaGetLastError());
  if (n_rows > 0) {
    kur_obs_kernel<<<(unsigned)((n_rows + 7) / 8), 256, 0, s>>>(rbuf, n_rows, k->R, r->n_begin, r->n_end,
                                                                 k->M, k->dt, *obs);
    SDE_CUDA_TRY(cudaGetLastError());
  }
  *rows = n_rows;
  return SDE_OK;
}

sde_status kuramoto_coupling(KuramotoCtx *k, const float *phi_dev, float *out_dev, cudaStream_t s) {
  SDE_CHECK_ARG(phi_dev != nullptr && out_dev != nullptr, "phi and out must be non-NULL");
  const int64_t NR = k->N * k->R;
  const int cvt_grid = (int)std::min<int64_t>((NR + 255) / 256, 4096);
  kur_to_fixed<<<cvt_grid, 256, 0, s>>>(phi_dev, k->theta, NR);
  SDE_CUDA_TRY(cudaGetLastError());
  if (k->model == SDE_KURAMOTO_GENERAL || k->model == SDE_KURAMOTO_GENERAL_FP32)
    return kuramoto_general_coupling(k, out_dev, s);
  const dim3 grid((unsigned)((k->N + 255) / 256), (unsigned)k->R);
  kur_coupling_uniform_kernel<<<grid, 256, 0, s>>>(k->theta, out_dev, k->N, (float)(k->K / (double)k->N));
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}

cudaError_t kur_order_launch(const uint32_t *theta, int64_t N, int64_t R, double *r_out, cudaStream_t s) {
  kur_order_kernel<<<(unsigned)R, 256, 0, s>>>(theta, N, R, r_out);
  return cudaGetLastError();
}

}  // namespace sde
