// tc_gemm_sk.cuh -- the general-coupling GEMM of tc_gemm.cuh with its K
// range split evenly over every CTA of the grid (stream-K), for products
// whose whole 128 x 256 tiles would leave most SMs idle (64 tiles on 152 SMs
// at N = 8192 and 128 replicas).  A K slice here costs about 1.4 times one
// of the whole-tile GEMMs, whose CTAs all read the same K slice of B (and
// pairs of them the same slice of A) at the same time; here the CTAs read
// at unrelated K offsets (measured: the same 805 MB into shared memory, L2
// throughput 57 % instead of 33 %, the tensor pipe 55 % instead of 74 % of
// the active cycles), so the split is selected only on request.
//
// The units of work are the (tile, K slice) pairs, tile-major (t = tile row
// * tiles_n + tile column, so that the two tiles of a tile row, which read
// the same rows of A, are worked on at the same time by neighbouring CTAs).
// CTA c takes the units [T c / P, T (c + 1) / P) of the T units: a run of
// segments, each the K slices [kb0, kb1) of one tile.  Only the first
// segment of a CTA can start inside a tile ("partial" segment: its FP32
// partial sums go to the CTA's workspace slot, then a flag carrying the
// launch's epoch is released); every other segment starts at K slice 0
// ("head" segment: its CTA adds the partial sums of the CTAs c + 1, c + 2, ...
// that cover the rest of the tile, after acquiring their flags, and runs the
// epilogue of the tile).  A CTA processes its partial segment first and any
// head segment last, so a head waits only for CTAs that started on its tile
// at the same time; with every CTA of the grid resident at once (the host
// sizes the grid so) every wait ends.  The sum of a tile is the head's
// accumulator plus the partials in CTA order: deterministic for a given grid
// size, equal to the one-pass GEMM up to FP32 rounding of the partial sums.
//
// Warp roles (320 threads):
//   warp 0, one thread : TMA producer over all units of the CTA (4-slot ring
//                        of 48 KB: A 128 x 64 and B 256 x 64, 128B swizzle)
//   warp 1, one thread : tcgen05.mma issuer (M = 128, N = 256, K = 16) into
//                        two TMEM accumulators of 256 columns, alternating per
//                        segment, so that one segment's epilogue runs while
//                        the next segment's MMAs accumulate
//   warps 2..9         : epilogue; warp w reads TMEM lane quarter w % 4 and
//                        column half (w - 2) / 4
// Every mbarrier wait and flag poll is bounded (a kernel argument, one second
// by default); on expiry the CTA records kErrTimeout, stops issuing, waits
// (with the fixed bound) for its own loads and MMAs in flight, frees its
// tensor memory and returns.
#pragma once

#include "tc_gemm.cuh"

namespace sde {
namespace tc {

constexpr int SK_BN = 256;
constexpr int SK_STAGES = 4;
constexpr int SK_EPI_WARPS = 8;
constexpr int SK_THREADS = 32 * (2 + SK_EPI_WARPS);
constexpr int SK_A_BYTES = BM * BK * 2;
constexpr int SK_B_BYTES = SK_BN * BK * 2;
constexpr int SK_STAGE_BYTES = SK_A_BYTES + SK_B_BYTES;
constexpr int SK_SMEM_BYTES = SK_STAGES * SK_STAGE_BYTES + 1024;
constexpr int SK_TMEM_COLS = 2 * SK_BN;  // two accumulators
constexpr int SK_COLS = SK_BN / 2;       // columns per epilogue thread
// fewest K slices a CTA should get (the host caps the grid at T / this)
constexpr int SK_MIN_UNITS = 16;

// First unit of CTA c of P over T units.
__device__ __forceinline__ int64_t sk_begin(int64_t T, int P, int c) { return T * (int64_t)c / (int64_t)P; }

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the epilogue warps only (named barrier 1).
__device__ __forceinline__ void epi_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * SK_EPI_WARPS) : "memory");
}

// The same barrier, returning to every epilogue thread whether any of them
// passed `cond` true: decisions to stop stay uniform across the epilogue
// warps (a thread that left while the others wait at a barrier would hang
// them).
__device__ __forceinline__ bool epi_any(bool cond) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)cond), "n"(32 * SK_EPI_WARPS)
      : "memory");
  return r != 0;
}

// One segment: the K slices [kb0, kb1) of tile t.
struct SkSeg {
  int t, kb0, kb1;
};

__device__ __forceinline__ SkSeg sk_segment(int64_t u, int64_t u_end, int nk) {
  SkSeg g;
  g.t = (int)(u / nk);
  g.kb0 = (int)(u % nk);
  const int64_t left = u_end - u;
  g.kb1 = (int)((int64_t)(nk - g.kb0) < left ? nk : g.kb0 + left);
  return g;
}

// D = A * B^T over K = Kdim with P = gridDim.x CTAs.  tiles_n = Ncols / 256,
// T = (M / 128) tiles_n (Kdim / 64).  ws: P slots of 256 x 128 FP32 (column
// major within the tile: [col][row]); flags: P words, zero at allocation,
// flag c = epoch once slot c holds this launch's partial.
template <int EPI>
__global__ void __launch_bounds__(SK_THREADS, 1)
    tc_gemm_sk_bf16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                           float *__restrict__ Dt, int M, int Kdim, int tiles_n, int64_t T, float *__restrict__ ws,
                           uint32_t *flags, uint32_t epoch, uint32_t *err, const StageArgs sa, uint64_t wait_ns) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *smA = smem;
  uint8_t *smB = smem + SK_STAGES * SK_A_BYTES;
  __shared__ __align__(8) uint64_t full_bar[SK_STAGES];
  __shared__ __align__(8) uint64_t empty_bar[SK_STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];  // accumulator b holds a finished segment
  __shared__ __align__(8) uint64_t acce_bar[2];  // the epilogue is done reading accumulator b
  __shared__ __align__(8) uint64_t done_bar;     // every MMA issued has completed
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x, P = gridDim.x;
  const int nk = Kdim / BK;
  const int64_t u_begin = sk_begin(T, P, c), u_end = sk_begin(T, P, c + 1);

  if (threadIdx.x == 0) {
    for (int s = 0; s < SK_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], SK_EPI_WARPS);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"((uint32_t)SK_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem = tmem_slot;
  griddep_wait();
  griddep_launch_dependents();

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer: every unit of the CTA, in order ----
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
      const uint64_t pol_a = l2_evict_first_policy();
      int issued = 0;
      for (int64_t u = u_begin; u < u_end; ++u) {
        const int it = (int)(u - u_begin);
        const int s = it % SK_STAGES;
        const uint32_t ph = (uint32_t)(it / SK_STAGES) & 1u;
        const int t = (int)(u / nk), kb = (int)(u % nk);
        if (!mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wait_ns)) break;
        mbar_arrive_expect_tx(&full_bar[s], (uint32_t)SK_STAGE_BYTES);
        tma_load_2d_hint(smA + s * SK_A_BYTES, &mapA, &full_bar[s], kb * BK, (t / tiles_n) * BM, pol_a);
        tma_load_2d(smB + s * SK_B_BYTES, &mapB, &full_bar[s], kb * BK, (t % tiles_n) * SK_BN);
        issued = it + 1;
      }
      // own loads land before the CTA may leave (older ones were consumed)
      volatile int no_abort = 0;
      for (int it = issued - SK_STAGES < 0 ? 0 : issued - SK_STAGES; it < issued; ++it)
        mbar_wait(&full_bar[it % SK_STAGES], (uint32_t)(it / SK_STAGES) & 1u, &no_abort);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: one accumulator per segment, alternating ----
      constexpr uint32_t idesc = idesc_bf16_f32(BM, SK_BN);
      int it = 0, seg = 0;
      bool alive = true;
      for (int64_t u = u_begin; u < u_end && alive; ++seg) {
        const SkSeg g = sk_segment(u, u_end, nk);
        const int b = seg & 1;
        // the epilogue of segment seg - 2 has read this accumulator out
        if (seg >= 2 && !mbar_wait(&acce_bar[b], (uint32_t)((seg >> 1) - 1) & 1u, &abort_flag, wait_ns)) break;
        tmem_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * SK_BN);
        for (int kb = g.kb0; kb < g.kb1; ++kb, ++it) {
          const int s = it % SK_STAGES;
          const uint32_t ph = (uint32_t)(it / SK_STAGES) & 1u;
          if (!mbar_wait(&full_bar[s], ph, &abort_flag, wait_ns)) {
            alive = false;
            break;
          }
          tmem_fence_after();
          const uint64_t adesc = smem_desc_sw128(smA + s * SK_A_BYTES);
          const uint64_t bdesc = smem_desc_sw128(smB + s * SK_B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / UMMA_K; ++k)
            umma_bf16(d, adesc + (uint64_t)(k * UMMA_K * 2 / 16), bdesc + (uint64_t)(k * UMMA_K * 2 / 16), idesc,
                      (kb != g.kb0 || k != 0) ? 1u : 0u);
          umma_commit(&empty_bar[s]);
        }
        umma_commit(&accf_bar[b]);  // (after an expiry the epilogue sees the abort flag)
        u += g.kb1 - g.kb0;
      }
      umma_commit(&done_bar);
      volatile int no_abort = 0;
      mbar_wait(&done_bar, 0, &no_abort);
    }
  } else {
    // ---- epilogue warps ----
    const int q = warp & 3;             // TMEM lane quarter
    const int h = (warp - 2) >> 2;      // column half
    const int row_l = q * 32 + lane;    // row within the tile
    const uint32_t lane_base = (uint32_t)((q * 32) << 16);
    const uint2 key = seed_to_key(sa.seed);
    int seg = 0;
    for (int64_t u = u_begin; u < u_end; ++seg) {
      const SkSeg g = sk_segment(u, u_end, nk);
      u += g.kb1 - g.kb0;
      const int b = seg & 1;
      const int m0 = (g.t / tiles_n) * BM, n0 = (g.t % tiles_n) * SK_BN;
      const bool got = mbar_wait(&accf_bar[b], (uint32_t)(seg >> 1) & 1u, &abort_flag, wait_ns);
      if (epi_any(!got || abort_flag)) break;
      tmem_fence_after();
      const uint32_t acc = tmem + lane_base + (uint32_t)(b * SK_BN + h * SK_COLS);
      if (g.kb0 != 0) {
        // partial segment: FP32 partial sums to this CTA's slot, then the flag
        float *slot = ws + (size_t)c * SK_BN * BM;
#pragma unroll 1
        for (int cc = 0; cc < SK_COLS; cc += 32) {
          float v[32];
          tmem_ld32(acc + (uint32_t)cc, v);
          const int col = h * SK_COLS + cc;
#pragma unroll
          for (int k = 0; k < 32; ++k) slot[(size_t)(col + k) * BM + row_l] = v[k];
        }
        __threadfence();
        epi_sync();
        if (threadIdx.x == 64) st_release_u32(flags + c, epoch);
      } else {
        // head segment: the CTAs after this one that start inside tile t
        int qn = 0;
        while (c + 1 + qn < P && sk_begin(T, P, c + 1 + qn) < (int64_t)(g.t + 1) * nk) ++qn;
        if (qn > 0) {
          if (threadIdx.x == 64) {
            const uint64_t t0 = globaltimer();
            for (int j = 1; j <= qn; ++j)
              while (ld_acquire_u32(flags + c + j) != epoch) {
                if (abort_flag) break;
                if (globaltimer() - t0 > wait_ns) {
                  abort_flag = 1;
                  break;
                }
              }
          }
          if (epi_any(abort_flag)) break;
        }
        const int row = m0 + row_l;
#pragma unroll 1
        for (int cc = 0; cc < SK_COLS; cc += 32) {
          float v[32];
          tmem_ld32(acc + (uint32_t)cc, v);
          const int col = h * SK_COLS + cc;
          for (int j = 1; j <= qn; ++j) {
            const float *slot = ws + (size_t)(c + j) * SK_BN * BM;
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] += slot[(size_t)(col + k) * BM + row_l];
          }
          if (EPI == EPI_STORE_D) {
#pragma unroll
            for (int k = 0; k < 32; ++k) Dt[(size_t)(n0 + col + k) * (size_t)M + row] = v[k];
          } else {
            stage_group<EPI == EPI_STAGE0 ? 0 : 1, 16>(sa, (int64_t)((n0 + col) / 2), (int64_t)row, v, key);
          }
        }
      }
      tmem_fence_before();
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acce_bar[b])) : "memory");
    }
  }
  __syncwarp();
  tmem_fence_before();
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)SK_TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && abort_flag) atomicOr(err, kErrTimeout);
}

}  // namespace tc
}  // namespace sde
