// mlp_tc.cuh -- forward pass of the surrogate network with its square hidden
// layers on the 5th-generation tensor cores (tcgen05), fused into one kernel.
//
// Network (width H = 256): h_0 = SiLU(x W_0^T + b_0) with x the n_in
// features, h_l = SiLU(h_{l-1} W_l^T + b_l) for the n_hh square layers,
// out = h_last . w_out + b_out.  Every product reads BF16 operands (weights
// and activations rounded from FP32) and accumulates in FP32, as the CUDA-core
// kernels of the training path do.
//
// One CTA takes 128 points (one tcgen05 M = 128 tile) of one ensemble member:
//   warps 0-15 (512 threads): layer 0 on the CUDA cores, then after each
//     square layer its epilogue -- tcgen05.ld of the FP32 accumulators, +
//     bias, SiLU, BF16 -- written back into shared memory as the next layer's
//     A operand in the 128-byte-swizzled K-major layout the MMA reads, or,
//     after the last square layer, the output dot product; warp w owns TMEM
//     lane quarter w % 4 (its 32 rows) and column quarter w / 4 (64
//     columns); the element arithmetic runs on packed FP32 pairs;
//   warp 16, one thread: TMA producer streaming the BF16 square-layer weights
//     through a 4-slot ring of 256 x 64 chunks (K-major, 128-byte swizzle);
//   warp 17, one thread: MMA issuer, M = 128, N = 256, K = 16 per
//     instruction, the accumulator (256 FP32 columns) in tensor memory, which
//     warp 17 allocates and frees.
// Layer handoffs go through mbarriers: `abuf` (512 arrivals: the A operand of
// the next square layer is in shared memory) and `acc` (tcgen05.commit: the
// accumulator is complete).  Every wait is bounded by one second of
// %globaltimer; on expiry the CTA stops, drains what it issued, records
// kErrTimeout and writes no output.
//
// SiLU(z) = z sigma(z), sigma(z) = 1 / (1 + 2^(-z log2 e)): the exponential
// by the hardware base-2 exponential (z clamped at -30), the reciprocal by
// two Newton steps from the initial guess as_float(0x7EF311C0 - as_int(y)),
// whose largest relative error on [1, oo) is 5.1% (the constant minimises it;
// searched for this library), so sigma is within ~1e-5 relative: below the
// BF16 rounding of the activations that follows.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace sde {
namespace mlptc {

constexpr int H = 256;             // hidden width
constexpr int BM = 128;            // points per CTA
constexpr int KCH = H / 64;        // 64-element K chunks per square layer
constexpr int A_CHUNK = BM * 128;  // bytes of one A chunk: 128 rows x 128 B
constexpr int W_CHUNK = H * 128;   // bytes of one weight chunk: 256 rows x 128 B
constexpr int RING = 4;            // weight chunks in flight
constexpr int EPI_WARPS = 16;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int PROD_WARP = EPI_WARPS;
constexpr int MMA_WARP = EPI_WARPS + 1;
constexpr int THREADS = EPI_THREADS + 64;
constexpr int SMEM_BYTES = KCH * A_CHUNK + RING * W_CHUNK + 1024;  // + alignment slack
constexpr int COLS_PER_WARP = H / (EPI_WARPS / 4);  // 64
constexpr int MAX_IN = 8;
constexpr int MAX_HH = 7;

struct Args {
  const float *X;       // [B][n_in] features
  const float *params;  // [members][P] FP32 master parameters
  int64_t P;
  int64_t B;
  int32_t n_in, n_hh;  // n_hh square layers (the hidden layers after the first)
  int64_t off_w0, off_b0, off_wo, off_bo;  // layer 0 and the output layer
  int64_t off_bh[MAX_HH];                  // biases of the square layers
  float *out;                              // [members][out_stride]
  int64_t out_stride;
  uint32_t *err;
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// SiLU of two values on packed FP32 pairs (the exponentials one at a time).
__device__ __forceinline__ float2 silu2(float2 z) {
  const float2 a = __fmul2_rn(make_float2(fmaxf(z.x, -30.0f), fmaxf(z.y, -30.0f)), f2(-1.44269504088896341f));
  float ex, ey;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ex) : "f"(a.x));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ey) : "f"(a.y));
  const float2 y = __fadd2_rn(make_float2(ex, ey), f2(1.0f));
  float2 r = make_float2(__int_as_float(0x7EF311C0 - __float_as_int(y.x)),
                         __int_as_float(0x7EF311C0 - __float_as_int(y.y)));
  const float2 ny = make_float2(-y.x, -y.y);
  r = __ffma2_rn(r, __ffma2_rn(ny, r, f2(1.0f)), r);
  r = __ffma2_rn(r, __ffma2_rn(ny, r, f2(1.0f)), r);
  return __fmul2_rn(z, r);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}

// Store 32 BF16 activations (16 packed pairs) of row m, columns n0..n0+31
// (n0 a multiple of 32), into the A buffer: K chunk n0 / 64, 16-byte units
// (n0 % 64) / 8 .. +3 of the row, each at position unit ^ (m % 8) (the
// 128-byte swizzle of the K-major layout).
__device__ __forceinline__ void store_row32(uint8_t *Ab, int m, int n0, const uint32_t (&p)[16]) {
  uint8_t *row = Ab + (n0 >> 6) * A_CHUNK + m * 128;
  const int j0 = (n0 & 63) >> 3;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int pos = (j0 + u) ^ (m & 7);
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(row + (pos << 4));
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(p[4 * u]), "r"(p[4 * u + 1]),
                 "r"(p[4 * u + 2]), "r"(p[4 * u + 3])
                 : "memory");
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(b)) : "memory");
}

__global__ void __launch_bounds__(THREADS, 1)
    mlp_fwd_tc_kernel(const __grid_constant__ CUtensorMap mapW, const Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *Ab = smem;                  // KCH chunks of [BM][128 B]
  uint8_t *Wr = smem + KCH * A_CHUNK;  // RING slots of [H][128 B]
  __shared__ __align__(16) float w0s[MAX_IN * H];  // [k][n]: output pairs adjacent
  __shared__ __align__(16) float b0s[H];
  __shared__ __align__(16) float bhs[MAX_HH * H];
  __shared__ __align__(16) float wos[H];
  __shared__ float part[EPI_WARPS / 4][BM];
  __shared__ __align__(8) uint64_t full_bar[RING];
  __shared__ __align__(8) uint64_t empty_bar[RING];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ __align__(8) uint64_t abuf_bar;
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int member = blockIdx.y;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  const float *pm = a.params + (int64_t)member * a.P;
  const int n_in = a.n_in, n_hh = a.n_hh;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RING; ++s) {
      tc::mbar_init(&full_bar[s], 1);
      tc::mbar_init(&empty_bar[s], 1);
    }
    tc::mbar_init(&acc_bar, 1);
    tc::mbar_init(&abuf_bar, EPI_THREADS);
    tc::mbar_init(&drain_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_addr(&tmem_slot)),
                 "r"((uint32_t)H)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // small parameters: layer 0 and the output weights BF16-rounded (the GEMM
  // operands), biases FP32
  for (int i = threadIdx.x; i < H * n_in; i += THREADS)  // W_0 is [n][k] in the parameters
    w0s[(i % n_in) * H + i / n_in] = bf16r(pm[a.off_w0 + i]);
  for (int i = threadIdx.x; i < H; i += THREADS) {
    b0s[i] = pm[a.off_b0 + i];
    wos[i] = bf16r(pm[a.off_wo + i]);
  }
  for (int i = threadIdx.x; i < n_hh * H; i += THREADS) bhs[i] = pm[a.off_bh[i / H] + (i % H)];
  const float bo = pm[a.off_bo];
  tc::tmem_fence_before();
  __syncthreads();
  tc::tmem_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == PROD_WARP) {
    if (lane == 0) {
      // ---- TMA producer: the square layers' weight chunks, in MMA order ----
      const int nchunks = n_hh * KCH;
      int issued = 0;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % RING;
        const uint32_t ph = (uint32_t)(c / RING) & 1u;
        if (!tc::mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) break;
        tc::mbar_arrive_expect_tx(&full_bar[s], (uint32_t)W_CHUNK);
        tc::tma_load_2d(Wr + s * W_CHUNK, &mapW, &full_bar[s], (c % KCH) * 64, (member * n_hh + c / KCH) * H);
        issued = c + 1;
      }
      // every load issued has landed before the CTA may end (older ones were
      // consumed by completed MMAs)
      volatile int no_abort = 0;
      for (int c = issued - RING < 0 ? 0 : issued - RING; c < issued; ++c)
        tc::mbar_wait(&full_bar[c % RING], (uint32_t)(c / RING) & 1u, &no_abort);
    }
    __syncwarp();
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      // ---- MMA issuer ----
      constexpr uint32_t idesc = tc::idesc_bf16_f32(BM, H);
      for (int l = 0; l < n_hh; ++l) {
        if (!tc::mbar_wait(&abuf_bar, (uint32_t)l & 1u, &abort_flag)) break;
        tc::tmem_fence_after();
        bool ok = true;
        for (int kc = 0; kc < KCH; ++kc) {
          const int c = l * KCH + kc;
          const int s = c % RING;
          if (!tc::mbar_wait(&full_bar[s], (uint32_t)(c / RING) & 1u, &abort_flag)) {
            ok = false;
            break;
          }
          tc::tmem_fence_after();
          const uint64_t adesc = tc::smem_desc_sw128(Ab + kc * A_CHUNK);
          const uint64_t bdesc = tc::smem_desc_sw128(Wr + s * W_CHUNK);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::umma_bf16(tmem, adesc + (uint64_t)(2 * k), bdesc + (uint64_t)(2 * k), idesc,
                          (kc | k) != 0 ? 1u : 0u);
          tc::umma_commit(&empty_bar[s]);
        }
        tc::umma_commit(&acc_bar);  // arrives once every MMA issued so far has completed
        if (!ok) break;
      }
      // every MMA issued has completed before the tensor memory is freed
      tc::umma_commit(&drain_bar);
      volatile int no_abort = 0;
      tc::mbar_wait(&drain_bar, 0u, &no_abort);
    }
    __syncwarp();
  } else {
    // ---- layer 0 and the epilogues: warps 0-15 ----
    const int q = warp & 3;   // TMEM lane quarter: rows 32 q .. 32 q + 31
    const int cq = warp >> 2; // column quarter: 64 cq .. 64 cq + 63
    const int m = q * 32 + lane;
    const int64_t row = row0 + m;
    const bool valid = row < a.B;
    float x[MAX_IN];
#pragma unroll
    for (int k = 0; k < MAX_IN; ++k) x[k] = (valid && k < n_in) ? bf16r(a.X[row * n_in + k]) : 0.0f;
#pragma unroll 1
    for (int g = 0; g < COLS_PER_WARP / 32; ++g) {
      const int n0 = cq * COLS_PER_WARP + g * 32;
      uint32_t p[16];
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        float2 z = *reinterpret_cast<const float2 *>(b0s + n0 + j);
#pragma unroll
        for (int k = 0; k < MAX_IN; ++k)
          if (k < n_in) z = __ffma2_rn(f2(x[k]), *reinterpret_cast<const float2 *>(w0s + k * H + n0 + j), z);
        const float2 h = silu2(z);
        p[j >> 1] = pack_bf16(h.x, h.y);
      }
      store_row32(Ab, m, n0, p);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive(&abuf_bar);
    float2 dot = make_float2(0.0f, 0.0f);
    bool done = n_hh == 0;
    for (int l = 0; l < n_hh; ++l) {
      if (!tc::mbar_wait(&acc_bar, (uint32_t)l & 1u, &abort_flag)) break;
      tc::tmem_fence_after();
      if (abort_flag) break;
      const bool last = l == n_hh - 1;
      const float *bl = bhs + l * H;
#pragma unroll 1
      for (int g = 0; g < COLS_PER_WARP / 32; ++g) {
        const int n0 = cq * COLS_PER_WARP + g * 32;
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)n0, v);
        if (!last) {
          uint32_t p[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const float2 h = silu2(__fadd2_rn(make_float2(v[j], v[j + 1]),
                                              *reinterpret_cast<const float2 *>(bl + n0 + j)));
            p[j >> 1] = pack_bf16(h.x, h.y);
          }
          store_row32(Ab, m, n0, p);
        } else {
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const float2 h = silu2(__fadd2_rn(make_float2(v[j], v[j + 1]),
                                              *reinterpret_cast<const float2 *>(bl + n0 + j)));
            dot = __ffma2_rn(make_float2(bf16r(h.x), bf16r(h.y)), *reinterpret_cast<const float2 *>(wos + n0 + j),
                             dot);
          }
        }
      }
      if (!last) {
        tc::tmem_fence_before();  // the accumulator is read before the next layer overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&abuf_bar);
      } else {
        done = true;
      }
    }
    // the four column quarters of each row
    part[cq][m] = dot.x + dot.y;
    asm volatile("bar.sync 1, %0;" ::"r"(EPI_THREADS) : "memory");
    if (cq == 0 && valid && done && !abort_flag)
      a.out[(int64_t)member * a.out_stride + row] = ((part[0][m] + part[1][m]) + (part[2][m] + part[3][m])) + bo;
  }
  tc::tmem_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)H)
                 : "memory");
  }
  if (threadIdx.x == 0 && abort_flag) atomicOr(a.err, kErrTimeout);
}

}  // namespace mlptc
}  // namespace sde
