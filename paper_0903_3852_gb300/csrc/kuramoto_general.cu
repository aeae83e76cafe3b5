// kuramoto_general.cu -- Eq. 2 with a general coupling matrix K_ij.
//
// The coupling sum is rewritten with sin(x_j - x_i) = sin x_j cos x_i -
// cos x_j sin x_i (the identity behind Eq. 3, applied row by row):
//
//   sum_j K_ij sin(x_j - x_i) = cos x_i P_s[i] - sin x_i P_c[i],
//   P_s = K sin(x),  P_c = K cos(x),
//
// so one SRK2 stage of all R replicas is one GEMM of K (N x N) with the
// 2R columns [sin x_r | cos x_r] plus an elementwise sub-step.  Two forms:
//   SDE_KURAMOTO_GENERAL      BF16 operands on tcgen05, FP32 accumulation in
//                             tensor memory (tc_gemm.cuh)
//   SDE_KURAMOTO_GENERAL_FP32 FP32 operands, FP32 CUDA-core GEMM (the
//                             baseline the tensor-core form is set against)
// Phases are 32-bit fixed-point turns as in kuramoto.cu; the receiving
// oscillator's own sin/cos are always evaluated in FP32 from its phase.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <utility>

#include "kuramoto.h"
#include "kuramoto_internal.h"
#include "philox.cuh"
#include "tc_gemm.cuh"
#include "tc_gemm_sk.cuh"
#include "tma_map.h"

namespace sde {

namespace {

template <typename T>
__device__ __forceinline__ T to_op(float v);
template <>
__device__ __forceinline__ float to_op<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// Operand rows [2r] = sin, [2r+1] = cos of every phase.  Grid: (N / 256, R).
template <typename T>
__global__ void kg_operand_kernel(const uint32_t *theta, T *op, int64_t N) {
  const int64_t r = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float s, c;
  sincos_turns(theta[r * N + i], s, c);
  op[(2 * r) * N + i] = to_op<T>(s);
  op[(2 * r + 1) * N + i] = to_op<T>(c);
}

// One SRK2 stage for every (replica, oscillator) from the GEMM output Dt
// (the forms without the fused epilogue): the same per-element update as the
// tensor-core epilogue (tc::stage_group), the next operand written as T.
// Grid: (N / 256, R).
// kStageIlp elements per thread (i, i + 256, ...): every input of the group is
// loaded before any arithmetic, so each thread keeps several loads in flight.
constexpr int kStageIlp = 4;

template <int STAGE, typename T>
__global__ void __launch_bounds__(256) kg_stage_kernel(const float *__restrict__ Dt, const tc::StageArgs a,
                                                       T *op_next) {
  const int64_t r = blockIdx.y;
  const int64_t N = a.N;
  const int64_t i0 = (int64_t)blockIdx.x * (256 * kStageIlp) + threadIdx.x;
  const uint2 key = seed_to_key(a.seed);
  uint32_t th[kStageIlp], th_s[kStageIlp];
  float ps[kStageIlp], pc[kStageIlp], om[kStageIlp], psi[kStageIlp], g1[kStageIlp];
  bool ok[kStageIlp];
#pragma unroll
  for (int u = 0; u < kStageIlp; ++u) {
    const int64_t i = i0 + u * 256;
    ok[u] = i < N;
    const int64_t ii = ok[u] ? i : 0;
    const int64_t idx = r * N + ii;
    ps[u] = Dt[(2 * r) * N + ii];
    pc[u] = Dt[(2 * r + 1) * N + ii];
    th[u] = a.theta[idx];
    th_s[u] = STAGE == 0 ? th[u] : a.theta_t[idx];
    om[u] = a.omega[idx];
    g1[u] = STAGE == 1 ? a.g1[idx] : 0.0f;
    psi[u] = (STAGE == 0 && a.fresh) ? 0.0f : tc::psi_plane(a, a.n >> 2, (int)(a.n & 3))[idx];
  }
#pragma unroll
  for (int u = 0; u < kStageIlp; ++u) {
    if (!ok[u]) continue;
    const int64_t i = i0 + u * 256;
    const int64_t idx = r * N + i;
    if (STAGE == 0 && a.fresh) psi[u] = tc::stage_noise<STAGE>(a, r, i, idx, key);
    const tc::StageOut o = tc::stage_math<STAGE>(a, th_s[u], th[u], om[u], psi[u], g1[u], ps[u], pc[u]);
    tc::stage_store<STAGE>(a, op_next, r, i, idx, o);
  }
}

// Coupling sums alone: out[r][i] = cos x_i Dt[2r][i] - sin x_i Dt[2r+1][i].
__global__ void kg_coupling_kernel(const float *__restrict__ Dt, const uint32_t *theta, float *out, int64_t N) {
  const int64_t r = blockIdx.y;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  float s, c;
  sincos_turns(theta[r * N + i], s, c);
  out[r * N + i] = c * Dt[(2 * r) * N + i] - s * Dt[(2 * r + 1) * N + i];
}

__global__ void kg_to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// ---- FP32 CUDA-core GEMM (baseline): Dt[c][i] = sum_j K[i][j] B[c][j] ----
// 128 x 128 tile per block of 256 threads, 8 x 8 outputs per thread, K
// slices of 8 staged (transposed) in shared memory, double buffered.
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

__global__ void __launch_bounds__(256) sgemm_nt_kernel(const float *__restrict__ A, const float *__restrict__ B,
                                                       float *__restrict__ Dt, int M, int Ncols, int Kdim) {
  __shared__ float As[2][SG_BK][SG_BM];
  __shared__ float Bs[2][SG_BK][SG_BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // 16 x 16 threads
  const int m0 = blockIdx.x * SG_BM, n0 = blockIdx.y * SG_BN;
  // loader mapping: 128 rows x 8 k = 256 float4: row = tid >> 1, k4 = (tid & 1) * 4
  const int lr = tid >> 1, lk = (tid & 1) * 4;
  const float *Ap = A + (size_t)(m0 + lr) * Kdim + lk;
  const float *Bp = B + (size_t)(n0 + lr) * Kdim + lk;
  const bool a_ok = (m0 + lr) < M, b_ok = (n0 + lr) < Ncols;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
  float4 ra = a_ok ? *(const float4 *)Ap : make_float4(0, 0, 0, 0);
  float4 rb = b_ok ? *(const float4 *)Bp : make_float4(0, 0, 0, 0);
  int buf = 0;
  As[0][lk + 0][lr] = ra.x;
  As[0][lk + 1][lr] = ra.y;
  As[0][lk + 2][lr] = ra.z;
  As[0][lk + 3][lr] = ra.w;
  Bs[0][lk + 0][lr] = rb.x;
  Bs[0][lk + 1][lr] = rb.y;
  Bs[0][lk + 2][lr] = rb.z;
  Bs[0][lk + 3][lr] = rb.w;
  __syncthreads();
  for (int k0 = 0; k0 < Kdim; k0 += SG_BK) {
    const bool more = k0 + SG_BK < Kdim;
    if (more) {
      ra = a_ok ? *(const float4 *)(Ap + k0 + SG_BK) : make_float4(0, 0, 0, 0);
      rb = b_ok ? *(const float4 *)(Bp + k0 + SG_BK) : make_float4(0, 0, 0, 0);
    }
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      float a[8], b[8];
      const float4 a0 = *(const float4 *)&As[buf][kk][ty * 4];
      const float4 a1 = *(const float4 *)&As[buf][kk][64 + ty * 4];
      const float4 b0 = *(const float4 *)&Bs[buf][kk][tx * 4];
      const float4 b1 = *(const float4 *)&Bs[buf][kk][64 + tx * 4];
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 8; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
    }
    if (more) {
      buf ^= 1;
      As[buf][lk + 0][lr] = ra.x;
      As[buf][lk + 1][lr] = ra.y;
      As[buf][lk + 2][lr] = ra.z;
      As[buf][lk + 3][lr] = ra.w;
      Bs[buf][lk + 0][lr] = rb.x;
      Bs[buf][lk + 1][lr] = rb.y;
      Bs[buf][lk + 2][lr] = rb.z;
      Bs[buf][lk + 3][lr] = rb.w;
      __syncthreads();
    }
  }
  // rows of this thread: m0 + {ty*4 .. ty*4+3, 64+ty*4 .. 64+ty*4+3}; columns likewise with tx
#pragma unroll
  for (int y = 0; y < 8; ++y) {
    const int col = n0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
    if (col >= Ncols) continue;
    float *dst = Dt + (size_t)col * M;
    const int r0 = m0 + ty * 4, r1 = m0 + 64 + ty * 4;
    if (r0 + 3 < M) *(float4 *)(dst + r0) = make_float4(acc[0][y], acc[1][y], acc[2][y], acc[3][y]);
    if (r1 + 3 < M) *(float4 *)(dst + r1) = make_float4(acc[4][y], acc[5][y], acc[6][y], acc[7][y]);
  }
}

constexpr int64_t kTimedStepStride = 8;

int grid_for(int64_t n, int sm_count) {
  const int64_t b = (n + 255) / 256;
  return (int)std::min<int64_t>(b, (int64_t)sm_count * 16);
}

// 2D BF16 tensor map: rows x cols (cols contiguous), box of box_rows x 64.
sde_status make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int box_rows) {
  return make_map_bf16(map, base, rows, cols, box_rows);
}

struct GemmPlan {
  CUtensorMap mapK;
  CUtensorMap mapOp[2];  // box of bn rows (one CTA's tile)
  CUtensorMap mapOpHalf[2];  // box of 128 rows (one CTA's half of a pair tile)
  int bn = 0;
  bool pair = false;  // CTA-pair GEMM (tc_gemm2_bf16_kernel)
  tc::EpiMaps em;     // pair GEMM: the SRK2 state its fused epilogue loads by TMA
  float *omega_copy = nullptr;  // [R][N] the run's omega (a fixed address for em.omega)
  // stream-K GEMM (tc_gemm_sk_bf16_kernel): sk_P CTAs, 0 = whole tiles
  int sk_P = 0;
  float *ws = nullptr;        // [sk_P][256][128] partial sums
  uint32_t *flags = nullptr;  // [sk_P] epoch of the partial in each slot
  uint32_t epoch = 0;
};

bool is_tc(const KuramotoCtx *k) { return k->model == SDE_KURAMOTO_GENERAL; }

void *op_buf(KuramotoCtx *k, int which) {
  if (is_tc(k)) return (void *)(k->Bt + (size_t)which * 2 * k->R * k->N);
  return (void *)(k->Bt32 + (size_t)which * 2 * k->R * k->N);
}

tc::StageArgs stage_args(KuramotoCtx *k, int next, const float *omega, int64_t n, int64_t run_begin) {
  const double inv2pi = 0.15915494309189533577;
  tc::StageArgs a{};
  a.theta = k->theta;
  a.theta_t = k->theta_t;
  a.g1 = k->g1;
  a.psi4 = k->psi4;
  a.omega = omega;
  a.op_next = (next >= 0 && is_tc(k)) ? (__nv_bfloat16 *)op_buf(k, next) : nullptr;
  a.N = k->N;
  a.NR = k->N * k->R;
  a.n = n;
  a.fresh = ((n & 3) == 0 || n == run_begin) ? 1 : 0;
  a.pre_slice = -1;
  a.wscale = (float)(k->dt * inv2pi);
  a.kc = (float)(k->dt * inv2pi);
  a.kh = (float)(0.5 * k->dt * inv2pi);
  a.sc = (float)(sqrt(2.0 * k->D * k->dt) * inv2pi);
  a.seed = k->seed;
  return a;
}

// Launch with programmatic stream serialization: the GEMM's prologue
// (barrier set-up, tensor-memory allocation) may start while the previous
// kernel of the stream finishes; the kernel waits (griddepcontrol.wait)
// before it reads anything that kernel wrote.
template <typename... Params, typename... Args>
cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, int threads, size_t smem, cudaStream_t s,
                             Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <int BN, int EPI>
cudaError_t launch_tc(KuramotoCtx *k, int which, const tc::StageArgs &sa, cudaStream_t s) {
  GemmPlan *g = (GemmPlan *)k->gemm_plan;
  const int M = (int)k->N, Ncols = (int)(2 * k->R), Kdim = (int)k->N;
  return launch_dependent(tc::tc_gemm_bf16_kernel<BN, EPI>, dim3(M / tc::BM, Ncols / BN), tc::EpiThreads<EPI>::value,
                          tc::Shape<BN>::SMEM_BYTES, s, g->mapK, g->mapOp[which], k->P, M, Kdim, k->err, sa,
                          k->wait_ns);
}

template <int EPI>
cudaError_t launch_tc2(KuramotoCtx *k, int which, const tc::StageArgs &sa, cudaStream_t s) {
  GemmPlan *g = (GemmPlan *)k->gemm_plan;
  const int M = (int)k->N, Ncols = (int)(2 * k->R), Kdim = (int)k->N;
  // clusters of two CTAs along x (the kernel's compile-time cluster shape)
  return launch_dependent(tc::tc_gemm2_bf16_kernel<EPI>, dim3(M / tc::BM, Ncols / tc::BN2),
                          tc::EpiThreads<EPI>::value, tc::SMEM2_BYTES, s, g->mapK, g->mapOpHalf[which], g->em, k->P,
                          M, Kdim, k->err, sa, k->wait_ns);
}

template <int EPI>
cudaError_t launch_sk(KuramotoCtx *k, int which, const tc::StageArgs &sa, cudaStream_t s) {
  GemmPlan *g = (GemmPlan *)k->gemm_plan;
  const int M = (int)k->N, Ncols = (int)(2 * k->R), Kdim = (int)k->N;
  const int tiles_n = Ncols / tc::SK_BN;
  const int64_t T = (int64_t)(M / tc::BM) * tiles_n * (Kdim / tc::BK);
  if (++g->epoch == 0) g->epoch = 1;  // flags start at 0: epoch 0 never marks a partial
  return launch_dependent(tc::tc_gemm_sk_bf16_kernel<EPI>, dim3((unsigned)g->sk_P), tc::SK_THREADS,
                          tc::SK_SMEM_BYTES, s, g->mapK, g->mapOp[which], k->P, M, Kdim, tiles_n, T, g->ws,
                          g->flags, g->epoch, k->err, sa, k->wait_ns);
}

// GEMM reading operand buffer `which`; epi = EPI_STORE_D writes Dt, the stage
// epilogues apply the SRK2 sub-step and write operand buffer 1 - which.
cudaError_t launch_gemm(KuramotoCtx *k, int which, cudaStream_t s, int epi = tc::EPI_STORE_D,
                        const float *omega = nullptr, int64_t n = 0, int64_t run_begin = 0) {
  const int M = (int)k->N, Ncols = (int)(2 * k->R), Kdim = (int)k->N;
  if (is_tc(k)) {
    GemmPlan *g = (GemmPlan *)k->gemm_plan;
    tc::StageArgs sa = stage_args(k, epi == tc::EPI_STORE_D ? -1 : 1 - which, omega, n, run_begin);
    if (g->pair && g->sk_P == 0 && epi != tc::EPI_STORE_D) {
      // the fused CTA-pair GEMMs of a Philox block draw the next block ahead,
      // a slice per launch; a block whose predecessor lay wholly in this run
      // is not drawn again at its first step
      const int64_t block = n >> 2;
      if (4 * block >= run_begin) sa.pre_slice = (int32_t)(2 * (n & 3) + (epi == tc::EPI_STAGE1 ? 1 : 0));
      if (block >= 1 && 4 * (block - 1) >= run_begin && n != run_begin) sa.fresh = 0;
    }
    if (g->sk_P > 0) {
      if (epi == tc::EPI_STAGE0) return launch_sk<tc::EPI_STAGE0>(k, which, sa, s);
      if (epi == tc::EPI_STAGE1) return launch_sk<tc::EPI_STAGE1>(k, which, sa, s);
      return launch_sk<tc::EPI_STORE_D>(k, which, sa, s);
    }
    if (g->pair) {
      if (epi == tc::EPI_STAGE0) return launch_tc2<tc::EPI_STAGE0>(k, which, sa, s);
      if (epi == tc::EPI_STAGE1) return launch_tc2<tc::EPI_STAGE1>(k, which, sa, s);
      return launch_tc2<tc::EPI_STORE_D>(k, which, sa, s);
    }
    if (g->bn == 256) {
      if (epi == tc::EPI_STAGE0) return launch_tc<256, tc::EPI_STAGE0>(k, which, sa, s);
      if (epi == tc::EPI_STAGE1) return launch_tc<256, tc::EPI_STAGE1>(k, which, sa, s);
      return launch_tc<256, tc::EPI_STORE_D>(k, which, sa, s);
    }
    if (epi == tc::EPI_STAGE0) return launch_tc<128, tc::EPI_STAGE0>(k, which, sa, s);
    if (epi == tc::EPI_STAGE1) return launch_tc<128, tc::EPI_STAGE1>(k, which, sa, s);
    return launch_tc<128, tc::EPI_STORE_D>(k, which, sa, s);
  } else {
    dim3 grid((M + SG_BM - 1) / SG_BM, (Ncols + SG_BN - 1) / SG_BN);
    sgemm_nt_kernel<<<grid, 256, 0, s>>>(k->Kf32, (const float *)op_buf(k, which), k->P, M, Ncols, Kdim);
  }
  return cudaGetLastError();
}

dim3 grid_nr(const KuramotoCtx *k) { return dim3((unsigned)((k->N + 255) / 256), (unsigned)k->R); }
dim3 grid_stage(const KuramotoCtx *k) {
  return dim3((unsigned)((k->N + 256 * kStageIlp - 1) / (256 * kStageIlp)), (unsigned)k->R);
}

cudaError_t launch_operand(KuramotoCtx *k, int which, cudaStream_t s) {
  if (is_tc(k))
    kg_operand_kernel<__nv_bfloat16><<<grid_nr(k), 256, 0, s>>>(k->theta, (__nv_bfloat16 *)op_buf(k, which),
                                                                 k->N);
  else
    kg_operand_kernel<float><<<grid_nr(k), 256, 0, s>>>(k->theta, (float *)op_buf(k, which), k->N);
  return cudaGetLastError();
}

template <int STAGE>
cudaError_t launch_stage(KuramotoCtx *k, int next, const float *omega, int64_t n, int64_t run_begin,
                         cudaStream_t s) {
  const tc::StageArgs a = stage_args(k, next, omega, n, run_begin);
  if (is_tc(k))
    kg_stage_kernel<STAGE, __nv_bfloat16><<<grid_stage(k), 256, 0, s>>>(k->P, a, (__nv_bfloat16 *)op_buf(k, next));
  else
    kg_stage_kernel<STAGE, float><<<grid_stage(k), 256, 0, s>>>(k->P, a, (float *)op_buf(k, next));
  return cudaGetLastError();
}

}  // namespace

sde_status kuramoto_general_alloc(KuramotoCtx *k) {
  const size_t NR = (size_t)k->N * (size_t)k->R;
  const size_t NN = (size_t)k->N * (size_t)k->N;
  if (is_tc(k)) {
    if (k->N % tc::BM != 0 || (2 * k->R) % 128 != 0) {
      set_error("invalid argument: the tensor-core form needs n_osc % 128 == 0 and n_replicas % 64 == 0 "
                "(use SDE_KURAMOTO_GENERAL_FP32 for other sizes)");
      return SDE_ERR_INVALID_ARG;
    }
  }
  if (!is_tc(k) && k->N % 8 != 0) {
    set_error("invalid argument: the FP32 general-coupling form needs n_osc % 8 == 0");
    return SDE_ERR_INVALID_ARG;
  }
  cudaError_t e;
  if ((e = device_alloc((void **)&k->theta_t, NR * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if ((e = device_alloc((void **)&k->g1, NR * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if ((e = device_alloc((void **)&k->P, NR * 2 * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if ((e = device_alloc((void **)&k->psi4, NR * 8 * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if (is_tc(k)) {
    if ((e = device_alloc((void **)&k->Kbf16, NN * 2)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = device_alloc((void **)&k->Bt, NR * 2 * 2 * 2)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    GemmPlan *g = new GemmPlan();
    k->gemm_plan = g;
    g->bn = (2 * k->R) % 256 == 0 ? 256 : 128;
    g->pair = k->N % 256 == 0 && (2 * k->R) % tc::BN2 == 0 && !(k->flags & SDE_FLAG_GEMM_SINGLE_CTA);
    sde_status st = make_map(&g->mapK, k->Kbf16, k->N, k->N, tc::BM);
    if (st != SDE_OK) return st;
    for (int w = 0; w < 2; ++w) {
      st = make_map(&g->mapOp[w], op_buf(k, w), 2 * k->R, k->N, g->bn);
      if (st != SDE_OK) return st;
      st = make_map(&g->mapOpHalf[w], op_buf(k, w), 2 * k->R, k->N, tc::BH2);
      if (st != SDE_OK) return st;
    }
    if (g->pair) {
      if ((e = device_alloc((void **)&g->omega_copy, NR * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      const struct {
        CUtensorMap *map;
        const void *base;
        int64_t planes;
      } arrays[] = {{&g->em.theta, k->theta, 1},   {&g->em.theta_t, k->theta_t, 1}, {&g->em.g1, k->g1, 1},
                    {&g->em.omega, g->omega_copy, 1}, {&g->em.psi, k->psi4, 8}};
      for (const auto &a : arrays) {
        st = make_map_w32(a.map, a.base, a.planes, k->R, k->N, tc::EQ_REPS, tc::BM);
        if (st != SDE_OK) return st;
      }
    }
    const void *kernels[] = {
        (const void *)tc::tc_gemm_bf16_kernel<256, tc::EPI_STORE_D>,
        (const void *)tc::tc_gemm_bf16_kernel<256, tc::EPI_STAGE0>,
        (const void *)tc::tc_gemm_bf16_kernel<256, tc::EPI_STAGE1>,
        (const void *)tc::tc_gemm_bf16_kernel<128, tc::EPI_STORE_D>,
        (const void *)tc::tc_gemm_bf16_kernel<128, tc::EPI_STAGE0>,
        (const void *)tc::tc_gemm_bf16_kernel<128, tc::EPI_STAGE1>};
    for (int q = 0; q < 6; ++q)
      if ((e = cudaFuncSetAttribute(kernels[q], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    q < 3 ? tc::Shape<256>::SMEM_BYTES : tc::Shape<128>::SMEM_BYTES)) !=
          cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
    const void *kernels2[] = {(const void *)tc::tc_gemm2_bf16_kernel<tc::EPI_STORE_D>,
                              (const void *)tc::tc_gemm2_bf16_kernel<tc::EPI_STAGE0>,
                              (const void *)tc::tc_gemm2_bf16_kernel<tc::EPI_STAGE1>};
    for (int q = 0; q < 3; ++q)
      if ((e = cudaFuncSetAttribute(kernels2[q], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tc::SMEM2_BYTES)) != cudaSuccess)
        return cuda_fail(e, "cudaFuncSetAttribute");
    // Stream-K on request (SDE_FLAG_GEMM_STREAM_K): as many CTAs as can be
    // resident at once (every CTA must be, for the heads' waits to end), each
    // with at least SK_MIN_UNITS K slices, where that is more CTAs than tiles.
    if (g->bn == 256 && (k->flags & SDE_FLAG_GEMM_STREAM_K)) {
      const void *kernels3[] = {(const void *)tc::tc_gemm_sk_bf16_kernel<tc::EPI_STORE_D>,
                                (const void *)tc::tc_gemm_sk_bf16_kernel<tc::EPI_STAGE0>,
                                (const void *)tc::tc_gemm_sk_bf16_kernel<tc::EPI_STAGE1>};
      int resident = 1 << 30;
      for (int q = 0; q < 3; ++q) {
        if ((e = cudaFuncSetAttribute(kernels3[q], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      tc::SK_SMEM_BYTES)) != cudaSuccess)
          return cuda_fail(e, "cudaFuncSetAttribute");
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernels3[q], tc::SK_THREADS,
                                                               tc::SK_SMEM_BYTES)) != cudaSuccess)
          return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        resident = std::min(resident, per_sm * k->sm_count);
      }
      const int64_t tiles = (k->N / tc::BM) * (2 * k->R / tc::SK_BN);
      const int64_t T = tiles * (k->N / tc::BK);
      const int64_t P = std::min<int64_t>(resident, T / tc::SK_MIN_UNITS);
      if (P > tiles) {
        g->sk_P = (int)P;
        if ((e = device_alloc((void **)&g->ws, (size_t)P * tc::SK_BN * tc::BM * sizeof(float))) != cudaSuccess)
          return cuda_fail(e, "cudaMalloc");
        if ((e = device_alloc((void **)&g->flags, (size_t)P * sizeof(uint32_t))) != cudaSuccess)
          return cuda_fail(e, "cudaMalloc");
        if ((e = cudaMemset(g->flags, 0, (size_t)P * sizeof(uint32_t))) != cudaSuccess)
          return cuda_fail(e, "cudaMemset");
      }
    }
  } else {
    if ((e = device_alloc((void **)&k->Kf32, NN * 4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    if ((e = device_alloc((void **)&k->Bt32, NR * 2 * 4 * 2)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  }
  k->block = is_tc(k) ? tc::THREADS : 256;
  k->opt = is_tc(k) ? ((GemmPlan *)k->gemm_plan)->bn : SG_BN;
  if (is_tc(k)) {
    const GemmPlan *g = (const GemmPlan *)k->gemm_plan;
    // CTAs per GEMM tile (0: stream-K, the split grid's CTA count in opt)
    k->cs = g->sk_P > 0 ? 0 : (g->pair ? 2 : 1);
    if (g->sk_P > 0) k->opt = g->sk_P;
  } else {
    k->cs = 1;
  }
  return SDE_OK;
}

void kuramoto_general_free(KuramotoCtx *k) {
  cudaFree(k->Kf32);
  cudaFree(k->Kbf16);
  cudaFree(k->Bt);
  cudaFree(k->Bt32);
  cudaFree(k->P);
  cudaFree(k->psi4);
  if (k->gemm_plan) {
    cudaFree(((GemmPlan *)k->gemm_plan)->ws);
    cudaFree(((GemmPlan *)k->gemm_plan)->flags);
    cudaFree(((GemmPlan *)k->gemm_plan)->omega_copy);
  }
  delete (GemmPlan *)k->gemm_plan;
  k->gemm_plan = nullptr;
}

sde_status kuramoto_set_coupling(KuramotoCtx *k, const float *K_dev, cudaStream_t s) {
  if (!(k->model == SDE_KURAMOTO_GENERAL || k->model == SDE_KURAMOTO_GENERAL_FP32)) {
    set_error("invalid argument: sde_set_coupling applies to the general-coupling models only");
    return SDE_ERR_INVALID_ARG;
  }
  SDE_CHECK_ARG(K_dev != nullptr, "K is NULL");
  const int64_t NN = k->N * k->N;
  if (is_tc(k)) {
    kg_to_bf16_kernel<<<grid_for(NN, k->sm_count), 256, 0, s>>>(K_dev, k->Kbf16, NN);
    SDE_CUDA_TRY(cudaGetLastError());
  } else {
    SDE_CUDA_TRY(cudaMemcpyAsync(k->Kf32, K_dev, sizeof(float) * NN, cudaMemcpyDeviceToDevice, s));
  }
  k->have_K = true;
  return SDE_OK;
}

sde_status kuramoto_general_run(KuramotoCtx *k, const sde_run_desc *r, cudaStream_t s, double *rbuf) {
  if (!k->have_K) {
    set_error("invalid argument: set the coupling matrix with sde_set_coupling before running");
    return SDE_ERR_INVALID_ARG;
  }
  SDE_CUDA_TRY(launch_operand(k, 0, s));
  // SDE_FLAG_TIME_KERNELS: an event between two GEMMs keeps the second one's
  // prologue from overlapping the first one's end, so the fused form (back
  // to back GEMMs, > 99 % of the loop) is timed as one block over all its
  // launches (the r(t) samples in between included), and the separate form
  // per GEMM launch on every kTimedStepStride-th step
  const bool fused = is_tc(k) && (k->flags & SDE_FLAG_FUSED);
  if (fused && ((GemmPlan *)k->gemm_plan)->pair && r->n_end > r->n_begin)
    SDE_CUDA_TRY(cudaMemcpyAsync(((GemmPlan *)k->gemm_plan)->omega_copy, r->omega_dev,
                                 sizeof(float) * (size_t)k->N * (size_t)k->R, cudaMemcpyDeviceToDevice, s));
  if (fused && r->n_end > r->n_begin) SDE_CUDA_TRY(ktime_begin(k, s));
  int64_t sample = 0;
  for (int64_t n = r->n_begin; n < r->n_end; ++n) {
    if (k->M > 0 && (n - r->n_begin) % k->M == 0) {
      SDE_CUDA_TRY(kur_order_launch(k->theta, k->N, k->R, rbuf + sample * k->R, s));
      ++sample;
    }
    if (fused) {
      // the SRK2 sub-steps run in the GEMM epilogues
      SDE_CUDA_TRY(launch_gemm(k, 0, s, tc::EPI_STAGE0, r->omega_dev, n, r->n_begin));
      SDE_CUDA_TRY(launch_gemm(k, 1, s, tc::EPI_STAGE1, r->omega_dev, n, r->n_begin));
      continue;
    }
    const bool timed = (n - r->n_begin) % kTimedStepStride == 0;
    if (timed) SDE_CUDA_TRY(ktime_begin(k, s));
    SDE_CUDA_TRY(launch_gemm(k, 0, s));
    if (timed) SDE_CUDA_TRY(ktime_end(k, s));
    SDE_CUDA_TRY(launch_stage<0>(k, 1, r->omega_dev, n, r->n_begin, s));
    if (timed) SDE_CUDA_TRY(ktime_begin(k, s));
    SDE_CUDA_TRY(launch_gemm(k, 1, s));
    if (timed) SDE_CUDA_TRY(ktime_end(k, s));
    SDE_CUDA_TRY(launch_stage<1>(k, 0, r->omega_dev, n, r->n_begin, s));
  }
  if (fused && r->n_end > r->n_begin) SDE_CUDA_TRY(ktime_end(k, s, 2 * (r->n_end - r->n_begin)));
  if (k->M > 0) SDE_CUDA_TRY(kur_order_launch(k->theta, k->N, k->R, rbuf + sample * k->R, s));
  return SDE_OK;
}

sde_status kuramoto_general_coupling(KuramotoCtx *k, float *out, cudaStream_t s) {
  if (!k->have_K) {
    set_error("invalid argument: set the coupling matrix with sde_set_coupling first");
    return SDE_ERR_INVALID_ARG;
  }
  SDE_CUDA_TRY(launch_operand(k, 0, s));
  SDE_CUDA_TRY(launch_gemm(k, 0, s));
  kg_coupling_kernel<<<grid_nr(k), 256, 0, s>>>(k->P, k->theta, out, k->N);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}

}  // namespace sde
