// tc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) for
// the general Kuramoto coupling of Eq. 2:
//
//   Dt[c][i] = sum_j K[i][j] * Bt[c][j],   Bt rows c = 2r (sin phi_r), 2r+1 (cos phi_r)
//
// so that sum_j K_ij sin(phi_j - phi_i) = cos(phi_i) Dt[2r][i] - sin(phi_i) Dt[2r+1][i].
// A = K (N x N, row i contiguous in j) and B = Bt (2R x N, row c contiguous in
// j) are both K-major; one CTA computes a 128 x BN tile of D with FP32
// accumulators in tensor memory:
//   warp 0, one thread : TMA producer (cp.async.bulk.tensor, 128B swizzle),
//                        STAGES-deep ring of (A, B) tiles guarded by mbarriers
//   warp 1, one thread : tcgen05.mma issuer (M = 128, N = BN, K = 16 per MMA),
//                        tcgen05.commit frees a ring slot / signals the end
//   all warps          : epilogue, tcgen05.ld 32x32b of their TMEM lane
//                        quarter, then either stores of Dt (each warp store
//                        is one 128 B row segment: the TMEM lane is the row
//                        index i) or the fused SRK2 sub-step (16 warps)
// The producer's and the MMA issuer's mbarrier waits are bounded by a limit
// in nanoseconds of %globaltimer (a kernel argument, one second by default);
// on expiry the CTA records kErrTimeout and stops issuing.  Whatever it did
// issue is then drained with waits of the fixed one-second bound, whatever
// the argument: the producer always waits for its last loads to land, and
// every thread waits for the commit that follows the last MMA, before the
// tensor memory is freed and the CTA returns.
//
// Two kernels: tc_gemm_bf16_kernel (one CTA per 128 x BN tile, described
// above) and tc_gemm2_bf16_kernel (one 256 x 256 tile per cluster of two
// CTAs, tcgen05 cta_group::2; its own notes below), the default where the
// sizes allow.  Both launch with programmatic dependent launch: their set-up
// runs before griddepcontrol.wait, everything the previous kernel wrote is
// read after it.  tc_gemm_sk.cuh holds the stream-K form.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "philox.cuh"
#include "turns.cuh"

namespace sde {
namespace tc {

constexpr int BM = 128;  // rows of D per CTA (MMA M)
constexpr int BK = 64;   // K elements per ring slot: one 128-byte swizzle row
constexpr int UMMA_K = 16;
constexpr int STAGES = 4;
constexpr int THREADS = 256;
constexpr uint64_t kTimeoutNs = 1000000000ull;

template <int BN>
struct Shape {
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;  // + alignment slack
  static constexpr int TMEM_COLS = BN;                            // FP32 accumulator columns
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}

// One try_wait: true once the phase of `parity` has completed; may suspend
// the thread for a while first.
__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok;
}

// The same test without suspending.
__device__ __forceinline__ uint32_t mbar_test_wait(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok;
}

// Wait for the phase of `parity` to complete; false if the CTA's abort flag
// is raised or limit_ns pass (then the flag is raised).  try_wait may
// suspend the thread longer than a short limit, so limits under a
// millisecond poll with test_wait.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort_flag,
                                          uint64_t limit_ns = kTimeoutNs) {
  const bool poll = limit_ns < 1000000ull;
  if (poll ? mbar_test_wait(b, parity) : mbar_try_wait(b, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (poll ? mbar_test_wait(b, parity) : mbar_try_wait(b, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > limit_ns) {
      *abort_flag = 1;
      return false;
    }
  }
}

// Address of the same shared-memory variable in the CTA of cluster rank
// `rank` (shared::cluster window).
__device__ __forceinline__ uint32_t mapa_shared(const void *p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
  return r;
}

// Count `bytes` as transferred on a local mbarrier's current phase without a
// transfer (for a share of a slot that will never be loaded).
__device__ __forceinline__ void mbar_complete_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ int ld_shared_cluster_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Programmatic dependent launch: wait until the grids this one depends on
// have completed and their memory is visible (a no-op for a plain launch),
// and let the next grid of the stream start its own prologue on free SMs.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster: arrive (release) and wait
// (acquire).  The forms without .aligned: threads of a warp may reach it
// from a bounded wait loop at different iterations.
__device__ __forceinline__ void cluster_barrier() {
  __syncwarp();
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// An L2 policy that evicts first what it tags: for the coupling matrix, which
// every GEMM streams once (read by the CTAs of one tile row at about the
// same time), so that it does not push the SRK2 state the epilogues read out
// of L2.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void tma_load_2d_hint(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                                 uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4}], [%2], %5;" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "l"(policy)
      : "memory");
}

// The same load for a CTA of a pair: the data lands in this CTA's shared
// memory, the byte count completes on the mbarrier at shared::cluster address
// `bar` (the even CTA's).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t bar, int c0,
                                                 int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, "
      "{%3, %4}], [%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_2d_pair_hint(void *dst, const CUtensorMap *map, uint32_t bar, int c0,
                                                      int c1, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2.L2::"
      "cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(bar), "r"(c0), "r"(c1), "l"(policy)
      : "memory");
}

// Shared-memory matrix descriptor of tcgen05 for a K-major tile written by
// TMA with 128-byte swizzling: rows of 128 bytes, 8-row groups 1024 bytes
// apart (stride byte offset), descriptor version 1, layout SWIZZLE_128B.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void *p) {
  const uint64_t addr = smem_addr(p);
  uint64_t d = (addr >> 4) & 0x3FFFull;
  d |= 1ull << 16;                  // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= 1ull << 46;                  // version
  d |= 2ull << 61;                  // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}

// The CTA-pair forms (cta_group::2): one MMA of M = 256 rows over the two
// CTAs of a pair, issued by the even CTA; each CTA supplies its own 128 rows
// of A and half of the N rows of B at the same shared-memory offsets as the
// issuer's descriptors, and receives its 128 rows of D in its own tensor
// memory at the same column address.
__device__ __forceinline__ void umma_bf16_pair(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                               uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// Arrive once on the mbarrier at this offset in both CTAs of the pair when
// every pair MMA issued before has completed.
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_addr(bar)),
      "h"((uint16_t)3)
      : "memory");
}

__device__ __forceinline__ void tmem_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Fused SRK2 sub-step of Eq. 2 in the epilogue (EPI_STAGE0 / EPI_STAGE1):
// the tile's column pairs (2r, 2r+1) are P_s, P_c of replica r for the row's
// oscillator i, so g = cos x_i P_s - sin x_i P_c is the coupling sum.
struct StageArgs {
  uint32_t *theta;     // [R][N] fixed-point turns
  uint32_t *theta_t;   // [R][N] predictor phases
  float *g1;           // [R][N] first-stage coupling sums
  float *psi4;         // [2][4][R][N] Gaussians of 4-step Philox blocks, one plane per step; block g in half g % 2
  const float *omega;  // [R][N]
  __nv_bfloat16 *op_next;  // [2R][N] operand of the next GEMM (the buffer this GEMM does not read)
  int64_t N;
  int64_t NR;     // N * R: plane stride of psi4
  int64_t n;      // step index
  int32_t fresh;  // stage 0: draw the Philox block of step n (its first step or the run's, unless drawn ahead)
  int32_t pre_slice;  // CTA-pair GEMM with the fused sub-step: draw slice pre_slice (0..7) of the next block
                      // while the MMAs run (the block's eight launches draw all of it); -1: none
  float wscale, kc, kh, sc;
  uint64_t seed;
};

enum { EPI_STORE_D = 0, EPI_STAGE0 = 1, EPI_STAGE1 = 2 };

// Plane q (the block's step q) of the Gaussians of Philox block `block`.
__device__ __forceinline__ float *psi_plane(const StageArgs &a, int64_t block, int q) {
  return a.psi4 + ((block & 1) * 4 + q) * a.NR;
}


// One element of a stage: oscillator i of replica r with coupling
// components ps = (K sin x)_i, pc = (K cos x)_i.  The Gaussians of a 4-step
// Philox block are drawn once (stage 0 of its first step in the run) and kept
// in four planes.  Shared by the fused epilogues and the separate stage
// kernels, so both give bit-identical phases.
__device__ __forceinline__ void store_operand(__nv_bfloat16 *op, int64_t idx, float v) {
  op[idx] = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void store_operand(float *op, int64_t idx, float v) { op[idx] = v; }

// The SRK2 sub-step of one element (replica r, oscillator i) from its loaded
// inputs: th_s the phase the coupling is taken at (theta for the predictor,
// theta~ for the corrector), th the current theta, the GEMM outputs (ps, pc),
// omega_i, the Gaussian psi and (corrector) the first-stage sum g1.  Shared
// by the separate stage kernel and the fused GEMM epilogue, so both compute
// bit for bit the same values.
struct StageOut {
  uint32_t out;  // theta~ (predictor) or the new theta (corrector)
  float g;       // this stage's coupling sum
  float so, co;  // sin, cos of `out`: the next GEMM operand
};

// The phase update of one element given sin / cos of the phase the coupling
// is taken at: g = cos x_i P_s - sin x_i P_c (its one rounding order fixed by
// the explicit FMA), then theta~ (predictor) or the new theta (corrector).
template <int STAGE>
__device__ __forceinline__ uint32_t stage_phase(const StageArgs &a, uint32_t th, float omega, float psi, float g1,
                                                float s, float c, float ps, float pc, float &g) {
  g = fmaf(c, ps, -(s * pc));
  const float wdt = omega * a.wscale;
  if (STAGE == 0) {
    const float d1 = fmaf(a.sc, psi, fmaf(a.kc, g, wdt));
    return th + (uint32_t)__float2int_rn(d1 * 4294967296.0f);
  }
  const float d = fmaf(a.sc, psi, fmaf(a.kh, g1 + g, wdt));
  return th + (uint32_t)__float2int_rn(d * 4294967296.0f);
}

template <int STAGE>
__device__ __forceinline__ StageOut stage_math(const StageArgs &a, uint32_t th_s, uint32_t th, float omega,
                                               float psi, float g1, float ps, float pc) {
  StageOut o;
  float s, c;
  sincos_turns(th_s, s, c);
  o.out = stage_phase<STAGE>(a, th, omega, psi, g1, s, c, ps, pc, o.g);
  sincos_turns(o.out, o.so, o.co);
  return o;
}

// The same for two elements at once, the sin/cos polynomials on packed FP32
// pairs (sincos_turns2: the same roundings as sincos_turns per element), so
// the results equal stage_math's bit for bit.
template <int STAGE>
__device__ __forceinline__ void stage_math2(const StageArgs &a, const uint32_t (&th_s)[2], const uint32_t (&th)[2],
                                            const float (&omega)[2], const float (&psi)[2], const float (&g1)[2],
                                            const float (&ps)[2], const float (&pc)[2], StageOut (&o)[2]) {
  float2 s, c;
  sincos_turns2(th_s[0], th_s[1], s, c);
  o[0].out = stage_phase<STAGE>(a, th[0], omega[0], psi[0], g1[0], s.x, c.x, ps[0], pc[0], o[0].g);
  o[1].out = stage_phase<STAGE>(a, th[1], omega[1], psi[1], g1[1], s.y, c.y, ps[1], pc[1], o[1].g);
  float2 so, co;
  sincos_turns2(o[0].out, o[1].out, so, co);
  o[0].so = so.x;
  o[0].co = co.x;
  o[1].so = so.y;
  o[1].co = co.y;
}

// The Gaussian of step n for element idx: drawn from the Philox block at the
// predictor of the block's first step (or of a run), which also keeps the
// block's later elements in psi4; read from psi4 otherwise.
template <int STAGE>
__device__ __forceinline__ float stage_noise(const StageArgs &a, int64_t r, int64_t i, int64_t idx, uint2 key) {
  const int q = (int)(a.n & 3);
  if (STAGE == 0 && a.fresh) {
    float zz[4];
    gauss4((uint32_t)(a.n >> 2), (uint32_t)i, (uint32_t)r, kTagKuramoto, key, zz);
    for (int k = q; k < 4; ++k) psi_plane(a, a.n >> 2, k)[idx] = zz[k];
    return pick4(zz, q);
  }
  return psi_plane(a, a.n >> 2, q)[idx];
}

template <int STAGE, typename T>
__device__ __forceinline__ void stage_store(const StageArgs &a, T *op_next, int64_t r, int64_t i, int64_t idx,
                                            const StageOut &o) {
  if (STAGE == 0) {
    a.theta_t[idx] = o.out;
    a.g1[idx] = o.g;
  } else {
    a.theta[idx] = o.out;
  }
  store_operand(op_next, (2 * r) * a.N + i, o.so);
  store_operand(op_next, (2 * r + 1) * a.N + i, o.co);
}

// NB consecutive replicas r0 .. r0 + NB - 1 of oscillator i, their coupling
// components in v[2j], v[2j + 1]: every input of the group is loaded before
// any arithmetic or store (the stores may alias the inputs as far as the
// compiler knows), so NB loads of each array are in flight at once.
template <int STAGE, int NB>
__device__ __forceinline__ void stage_group(const StageArgs &a, int64_t r0, int64_t i, const float *v, uint2 key) {
  uint32_t th[NB], th_s[NB];
  float om[NB], psi[NB], g1[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    const int64_t idx = (r0 + j) * a.N + i;
    th[j] = a.theta[idx];
    th_s[j] = STAGE == 0 ? th[j] : a.theta_t[idx];
    om[j] = a.omega[idx];
    g1[j] = STAGE == 1 ? a.g1[idx] : 0.0f;
    psi[j] = (STAGE == 0 && a.fresh) ? 0.0f : psi_plane(a, a.n >> 2, (int)(a.n & 3))[idx];
  }
  static_assert(NB % 2 == 0, "replicas in pairs");
#pragma unroll
  for (int j = 0; j < NB; j += 2) {
    const int64_t r = r0 + j, idx = r * a.N + i;
    if (STAGE == 0 && a.fresh) {
      psi[j] = stage_noise<STAGE>(a, r, i, idx, key);
      psi[j + 1] = stage_noise<STAGE>(a, r + 1, i, idx + a.N, key);
    }
    StageOut o[2];
    stage_math2<STAGE>(a, {th_s[j], th_s[j + 1]}, {th[j], th[j + 1]}, {om[j], om[j + 1]}, {psi[j], psi[j + 1]},
                       {g1[j], g1[j + 1]}, {v[2 * j], v[2 * j + 2]}, {v[2 * j + 1], v[2 * j + 3]}, o);
    stage_store<STAGE>(a, a.op_next, r, i, idx, o[0]);
    stage_store<STAGE>(a, a.op_next, r + 1, i, idx + a.N, o[1]);
  }
}

// Threads per CTA: 8 warps for the plain store, 16 for the fused stages
// (more warps to hide the latency of the per-element SRK2 arithmetic).
template <int EPI>
struct EpiThreads {
  static constexpr int value = EPI == EPI_STORE_D ? 256 : 512;
};

// Epilogue of one 128 x BN tile whose FP32 accumulators sit in this CTA's
// tensor memory (lane = row, column = column): warp w reads TMEM lane
// quarter w % 4 (the lanes it may access) and column group w / 4, then
// stores Dt or applies the SRK2 sub-step.
template <int BN, int EPI>
__device__ __forceinline__ void epilogue_tile(uint32_t tmem, int m0, int n0, float *__restrict__ Dt, int M,
                                              const StageArgs &sa) {
  constexpr int NGROUPS = EpiThreads<EPI>::value / 128;  // column groups of the epilogue
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3;       // TMEM lane quarter this warp may access
  const int group = warp >> 2;  // which BN / NGROUPS columns
  const int row = m0 + q * 32 + lane;
  const uint2 key = seed_to_key(sa.seed);
#pragma unroll 1
  for (int cc = 0; cc < BN / NGROUPS; cc += 32) {
    const int col = group * (BN / NGROUPS) + cc;
    float v[32];
    tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, v);
    if (EPI == EPI_STORE_D) {
#pragma unroll
      for (int i = 0; i < 32; ++i) Dt[(size_t)(n0 + col + i) * (size_t)M + row] = v[i];
    } else {
      // the chunk's 16 replicas in two groups of 8
      stage_group<EPI == EPI_STAGE0 ? 0 : 1, 8>(sa, (int64_t)((n0 + col) / 2), (int64_t)row, v, key);
      stage_group<EPI == EPI_STAGE0 ? 0 : 1, 8>(sa, (int64_t)((n0 + col) / 2 + 8), (int64_t)row, v + 16, key);
    }
  }
}

// D = A * B^T over K = Kdim.  EPI_STORE_D writes Dt transposed ([col][row],
// rows contiguous) so that each column of the tile is one coalesced run;
// the stage epilogues apply the SRK2 sub-step instead.
// Requires M % 128 == 0, Ncols % BN == 0, Kdim % 64 == 0 (checked by the host).
template <int BN, int EPI>
__global__ void __launch_bounds__(EpiThreads<EPI>::value, 1)
    tc_gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                        float *__restrict__ Dt, int M, int Kdim, uint32_t *err, const StageArgs sa,
                        uint64_t wait_ns) {
  using S = Shape<BN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *smA = smem;
  uint8_t *smB = smem + STAGES * S::A_BYTES;
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int nk = Kdim / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"((uint32_t)S::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem = tmem_slot;
  // everything above overlaps the previous kernel of the stream (programmatic
  // dependent launch); the operand and the SRK2 state are read only below
  griddep_wait();
  griddep_launch_dependents();

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
    const uint64_t pol_a = l2_evict_first_policy();
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wait_ns)) break;
      mbar_arrive_expect_tx(&full_bar[s], (uint32_t)S::STAGE_BYTES);
      tma_load_2d_hint(smA + s * S::A_BYTES, &mapA, &full_bar[s], kb * BK, m0, pol_a);
      tma_load_2d(smB + s * S::B_BYTES, &mapB, &full_bar[s], kb * BK, n0);
      issued = kb + 1;
    }
    {
      // Wait until this CTA's own loads have landed before anyone may free the
      // CTA: the MMA issuer can give up on a load after the last one was
      // issued.  Loads older than the last STAGES were consumed by MMAs that
      // completed (the producer waited for their slots), and on the normal
      // path these waits return at once.
      volatile int no_abort = 0;
      for (int kb = issued - STAGES < 0 ? 0 : issued - STAGES; kb < issued; ++kb)
        mbar_wait(&full_bar[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, &no_abort);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag, wait_ns)) break;
      tmem_fence_after();
      const uint64_t adesc = smem_desc_sw128(smA + s * S::A_BYTES);
      const uint64_t bdesc = smem_desc_sw128(smB + s * S::B_BYTES);
#pragma unroll
      for (int k = 0; k < BK / UMMA_K; ++k)
        umma_bf16(tmem, adesc + (uint64_t)(k * UMMA_K * 2 / 16), bdesc + (uint64_t)(k * UMMA_K * 2 / 16),
                  idesc, (kb | k) != 0 ? 1u : 0u);
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&acc_bar);  // arrives when every MMA issued above has completed
  }
  __syncwarp();

  // ---- epilogue: all warps ----
  volatile int no_abort = 0;
  const bool ok = mbar_wait(&acc_bar, 0, &no_abort) && !abort_flag;
  tmem_fence_after();
  if (ok) epilogue_tile<BN, EPI>(tmem, m0, n0, Dt, M, sa);
  tmem_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)S::TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && (abort_flag || !ok)) atomicOr(err, kErrTimeout);
}

// ---- CTA-pair GEMM (cta_group::2) --------------------------------------
//
// The same product with one 256 x 256 tile of D per pair of CTAs (a cluster
// of two along M).  Each CTA stages its own 128 rows of A and 128 of the 256
// rows of B per K slice (32 KB instead of 48 KB for 128 x 256 of D), so the
// shared-memory writes (TMA) and reads (MMA) per FLOP fall by a third.
//   both CTAs   : TMA producer for its own half of each slot; the bytes of
//                 both halves complete on the even CTA's full_bar
//   even CTA    : MMA issuer of the pair (M = 256, N = 256, K = 16 per MMA);
//                 tcgen05.commit multicasts every slot release (empty_bar)
//                 and the final accumulator barrier to both CTAs
//   all warps   : epilogue of this CTA's 128 rows from its own tensor memory
// Teardown: after the accumulator barrier a cluster barrier makes both CTAs'
// issue counts final; where a wait expired, the even CTA completes the phase
// of every slot loaded but not consumed (accounting for the half that was
// never issued) and waits for it, so that no load of either CTA is in flight
// when the final cluster barrier lets the CTAs free their tensor memory and
// leave.
constexpr int STAGES2 = 6;
constexpr int BN2 = 256;       // D columns per pair (both CTAs hold all of them)
constexpr int BH2 = BN2 / 2;   // B rows per CTA
constexpr int A2_BYTES = BM * BK * 2;
constexpr int B2_BYTES = BH2 * BK * 2;
constexpr int STAGE2_BYTES = A2_BYTES + B2_BYTES;  // one CTA's half of a slot
constexpr int SMEM2_BYTES = STAGES2 * STAGE2_BYTES + 1024;
constexpr int TMEM2_COLS = BN2;

// The SRK2 state an epilogue reads, as TMA tensor maps of 4-byte words over
// [R][N] (psi: the eight planes [2][4][R][N]), boxes of 128 oscillators x 32
// replicas.
struct EpiMaps {
  CUtensorMap theta, theta_t, g1, omega, psi;
};

constexpr int EQ_REPS = 32;                     // replicas per quarter of a tile
constexpr int EQ_ARR_BYTES = EQ_REPS * BM * 4;  // one array's box: 16 KB
constexpr int EQ_BUF_BYTES = 5 * EQ_ARR_BYTES;  // theta, omega, psi, theta~, g1
static_assert(2 * EQ_BUF_BYTES <= STAGES2 * STAGE2_BYTES, "epilogue inputs must fit in the ring");

// The fused SRK2 sub-step of the CTA-pair GEMM, after its MMAs: the inputs
// of the CTA's 128 oscillators x 128 replicas (theta, omega, the Gaussians
// and, for the corrector, theta~ and the first-stage sums) come into the now
// idle ring by TMA, a quarter of the replicas (32) at a time in two
// alternating buffers, so that one quarter loads while the previous one is
// finished.  Warp w: TMEM lane quarter w % 4 (its 32 oscillators), replicas
// 8 (w / 4) .. 8 (w / 4) + 7 of each quarter.  Thread 0 issues the loads; the
// buffer of quarter c is reloaded for quarter c + 2 once every warp has
// released it.  Same arithmetic as stage_group on the same values.
// A wait that expires (the fixed one-second bound) records kErrTimeout in
// *err: the quarter's results are then not to be trusted.
template <int EPI>
__device__ __forceinline__ void pair_stage_epilogue(uint32_t tmem, int m0, int n0, const StageArgs &sa,
                                                    const EpiMaps &em, uint8_t *smem, uint64_t *epi_full,
                                                    uint64_t *epi_free, uint32_t *err) {
  constexpr int STAGE = EPI == EPI_STAGE1 ? 1 : 0;
  constexpr int W = EQ_ARR_BYTES / 4;  // words per array box
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lq = warp & 3, grp = warp >> 2;
  const int row_l = lq * 32 + lane;
  const int64_t i = m0 + row_l;
  const int na = STAGE == 1 ? 5 : (sa.fresh ? 2 : 3);
  const uint2 key = seed_to_key(sa.seed);
  volatile int no_abort = 0;
  auto issue = [&](int c) {
    uint8_t *buf = smem + (c & 1) * EQ_BUF_BYTES;
    uint64_t *bar = &epi_full[c & 1];
    const int r0 = n0 / 2 + EQ_REPS * c;
    mbar_arrive_expect_tx(bar, (uint32_t)(na * EQ_ARR_BYTES));
    tma_load_2d(buf, &em.theta, bar, m0, r0);
    tma_load_2d(buf + EQ_ARR_BYTES, &em.omega, bar, m0, r0);
    if (na >= 3)
      tma_load_3d(buf + 2 * EQ_ARR_BYTES, &em.psi, bar, m0, r0, (int)(((sa.n >> 2) & 1) * 4 + (sa.n & 3)));
    if (STAGE == 1) {
      tma_load_2d(buf + 3 * EQ_ARR_BYTES, &em.theta_t, bar, m0, r0);
      tma_load_2d(buf + 4 * EQ_ARR_BYTES, &em.g1, bar, m0, r0);
    }
  };
  if (threadIdx.x == 0) {
    issue(0);
    issue(1);
  }
#pragma unroll 1
  for (int c = 0; c < BN2 / 2 / EQ_REPS; ++c) {
    if (!mbar_wait(&epi_full[c & 1], (uint32_t)(c >> 1) & 1u, &no_abort)) atomicOr(err, kErrTimeout);
    __syncwarp();
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(2 * EQ_REPS * c + 16 * grp), v);
    const uint32_t *buf = (const uint32_t *)(smem + (c & 1) * EQ_BUF_BYTES);
#pragma unroll
    for (int j = 0; j < 8; j += 2) {
      uint32_t th[2], th_s[2];
      float om[2], psi[2], g1[2];
      int64_t r[2], idx[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int rl = 8 * grp + j + h;  // replica within the quarter
        r[h] = n0 / 2 + EQ_REPS * c + rl;
        idx[h] = r[h] * sa.N + i;
        const int o = rl * BM + row_l;
        th[h] = buf[o];
        om[h] = __uint_as_float(buf[W + o]);
        psi[h] = (STAGE == 0 && sa.fresh) ? stage_noise<0>(sa, r[h], i, idx[h], key) : __uint_as_float(buf[2 * W + o]);
        th_s[h] = STAGE == 0 ? th[h] : buf[3 * W + o];
        g1[h] = STAGE == 1 ? __uint_as_float(buf[4 * W + o]) : 0.0f;
      }
      StageOut out[2];
      stage_math2<STAGE>(sa, th_s, th, om, psi, g1, {v[2 * j], v[2 * j + 2]}, {v[2 * j + 1], v[2 * j + 3]}, out);
      stage_store<STAGE>(sa, sa.op_next, r[0], i, idx[0], out[0]);
      stage_store<STAGE>(sa, sa.op_next, r[1], i, idx[1], out[1]);
    }
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&epi_free[c & 1])) : "memory");
    if (threadIdx.x == 0 && c + 2 < BN2 / 2 / EQ_REPS) {
      if (!mbar_wait(&epi_free[c & 1], (uint32_t)(c >> 1) & 1u, &no_abort)) atomicOr(err, kErrTimeout);
      // the buffer's last readers were generic loads; order them before the
      // TMA's writes
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(c + 2);
    }
  }
}

// D = A * B^T, tile rows m0 = 128 * blockIdx.x (the pair covers 256 rows),
// columns n0 = 256 * blockIdx.y.  mapB's box is 128 rows (half a tile).
// Requires M % 256 == 0, Ncols % 256 == 0, Kdim % 64 == 0 (checked by the
// host); launched with gridDim.x even (clusters of 2 along x).
template <int EPI>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(EpiThreads<EPI>::value, 1)
    tc_gemm2_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                         const __grid_constant__ EpiMaps em, float *__restrict__ Dt, int M, int Kdim, uint32_t *err,
                         const StageArgs sa, uint64_t wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *smA = smem;
  uint8_t *smB = smem + STAGES2 * A2_BYTES;
  __shared__ __align__(8) uint64_t full_bar[STAGES2];   // even CTA: both halves of the slot landed
  __shared__ __align__(8) uint64_t empty_bar[STAGES2];  // the pair's MMAs of the slot completed
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int issued_cnt;    // K slices whose loads this CTA issued
  __shared__ int consumed_cnt;  // even CTA: K slices whose MMAs were issued
  __shared__ __align__(8) uint64_t epi_full[2];  // SRK2 epilogue: a quarter's inputs landed
  __shared__ __align__(8) uint64_t epi_free[2];  // SRK2 epilogue: every warp is done with a buffer

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN2;
  const int nk = Kdim / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES2; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&epi_full[b], 1);
      mbar_init(&epi_free[b], EpiThreads<EPI>::value / 32);
    }
    abort_flag = 0;
    issued_cnt = 0;
    consumed_cnt = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    // one warp of each CTA of the pair allocates, together, the same columns
    // of both CTAs' tensor memory
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"((uint32_t)TMEM2_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  cluster_barrier();  // both CTAs' barriers initialised, tensor memory allocated
  tmem_fence_after();
  const uint32_t tmem = tmem_slot;
  // The coupling matrix (A) is written only before a run, so the first slots'
  // A loads may start while the previous kernel of the stream finishes; the
  // operand (B) and the SRK2 state are read only after griddepcontrol.wait.
  const int pre = nk < STAGES2 ? nk : STAGES2;
  const int b_row = n0 + (int)rank * BH2;
  uint64_t pol_a = 0;
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
    pol_a = l2_evict_first_policy();
    for (int kb = 0; kb < pre; ++kb) {  // fresh slots: nothing to wait for
      if (rank == 0) mbar_arrive_expect_tx(&full_bar[kb], 2u * (uint32_t)STAGE2_BYTES);
      tma_load_2d_pair_hint(smA + kb * A2_BYTES, &mapA, mapa_shared(&full_bar[kb], 0), kb * BK, m0, pol_a);
    }
  }
  griddep_wait();  // as in the one-CTA kernel
  griddep_launch_dependents();

  if (EPI != EPI_STORE_D && sa.pre_slice >= 0 && warp >= 2) {
    // The warps that wait for the accumulators draw a slice of the next
    // Philox block of this CTA's elements meanwhile: replicas 16 pre_slice ..
    // 16 pre_slice + 15 of the tile, all 128 oscillators, four Gaussians
    // each, into the other half of psi4 (its last readers were the previous
    // block's launches, which are complete).
    const uint32_t gnext = (uint32_t)(sa.n >> 2) + 1u;
    const uint2 key = seed_to_key(sa.seed);
#pragma unroll 1
    for (int e = (int)threadIdx.x - 64; e < 16 * BM; e += EpiThreads<EPI>::value - 64) {
      const int64_t r = n0 / 2 + 16 * sa.pre_slice + (e >> 7), i = m0 + (e & (BM - 1));
      const int64_t idx = r * sa.N + i;
      float zz[4];
      gauss4(gnext, (uint32_t)i, (uint32_t)r, kTagKuramoto, key, zz);
#pragma unroll
      for (int k = 0; k < 4; ++k) psi_plane(sa, gnext, k)[idx] = zz[k];
    }
  }

  if (warp == 0 && lane == 0) {
    // ---- TMA producer (both CTAs, each its own half) ----
    for (int kb = 0; kb < pre; ++kb)
      tma_load_2d_pair(smB + kb * B2_BYTES, &mapB, mapa_shared(&full_bar[kb], 0), kb * BK, b_row);
    int issued = pre;
    for (int kb = pre; kb < nk; ++kb) {
      const int s = kb % STAGES2;
      const uint32_t ph = (uint32_t)(kb / STAGES2) & 1u;
      if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wait_ns)) break;
      if (rank == 0) mbar_arrive_expect_tx(&full_bar[s], 2u * (uint32_t)STAGE2_BYTES);
      const uint32_t fb = mapa_shared(&full_bar[s], 0);
      tma_load_2d_pair_hint(smA + s * A2_BYTES, &mapA, fb, kb * BK, m0, pol_a);
      tma_load_2d_pair(smB + s * B2_BYTES, &mapB, fb, kb * BK, b_row);
      issued = kb + 1;
    }
    issued_cnt = issued;
  } else if (warp == 1 && lane == 0 && rank == 0) {
    // ---- MMA issuer of the pair ----
    constexpr uint32_t idesc = idesc_bf16_f32(2 * BM, BN2);
    int kb = 0;
    for (; kb < nk; ++kb) {
      const int s = kb % STAGES2;
      const uint32_t ph = (uint32_t)(kb / STAGES2) & 1u;
      if (!mbar_wait(&full_bar[s], ph, &abort_flag, wait_ns)) break;
      tmem_fence_after();
      const uint64_t adesc = smem_desc_sw128(smA + s * A2_BYTES);
      const uint64_t bdesc = smem_desc_sw128(smB + s * B2_BYTES);
#pragma unroll
      for (int k = 0; k < BK / UMMA_K; ++k)
        umma_bf16_pair(tmem, adesc + (uint64_t)(k * UMMA_K * 2 / 16), bdesc + (uint64_t)(k * UMMA_K * 2 / 16),
                       idesc, (kb | k) != 0 ? 1u : 0u);
      umma_commit_pair(&empty_bar[s]);
    }
    consumed_cnt = kb;
    umma_commit_pair(&acc_bar);  // arrives in both CTAs when every MMA issued above has completed
  }
  __syncwarp();

  volatile int no_abort = 0;
  const bool acc_ok = mbar_wait(&acc_bar, 0, &no_abort);
  cluster_barrier();  // issue counts, the consumed count and both abort flags are final
  const bool ok = acc_ok && !abort_flag && !ld_shared_cluster_s32(mapa_shared(&abort_flag, rank ^ 1u));
  if (rank == 0 && threadIdx.x == 0) {
    // Slots loaded but not consumed (after an expired wait only): at most
    // STAGES2 consecutive K slices, one per slot, each the slot's pending
    // phase.  A half issued by one CTA only: count the other half as done
    // (or make the arrival the even CTA never made), then wait for the phase.
    const int own = issued_cnt, peer = ld_shared_cluster_s32(mapa_shared(&issued_cnt, 1u));
    const int hi = own > peer ? own : peer;
    volatile int no_abort2 = 0;
    for (int kb = consumed_cnt; kb < hi; ++kb) {
      const int s = kb % STAGES2;
      if (kb < own && kb >= peer) mbar_complete_tx(&full_bar[s], (uint32_t)STAGE2_BYTES);
      if (kb >= own && kb < peer) mbar_arrive_expect_tx(&full_bar[s], (uint32_t)STAGE2_BYTES);
      mbar_wait(&full_bar[s], (uint32_t)(kb / STAGES2) & 1u, &no_abort2);
    }
  }
  // ---- epilogue: all warps of both CTAs, each CTA its own 128 rows ----
  tmem_fence_after();
  if (ok) {
    if (EPI == EPI_STORE_D)
      epilogue_tile<BN2, EPI>(tmem, m0, n0, Dt, M, sa);
    else
      pair_stage_epilogue<EPI>(tmem, m0, n0, sa, em, smem, epi_full, epi_free, err);
  }
  tmem_fence_before();
  // neither CTA frees the pair's tensor memory or leaves (with its barriers
  // and shared memory) while the other, or a load, may still use them
  cluster_barrier();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)TMEM2_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && (abort_flag || !ok)) atomicOr(err, kErrTimeout);
}

}  // namespace tc
}  // namespace sde
