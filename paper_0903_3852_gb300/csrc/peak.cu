// peak.cu -- FP32 fused-multiply-add throughput probe (measurement only).
//
// The FP32 roofline of the integration kernels is taken against a measured
// peak rather than the unit count times the nominal clock: every thread runs
// eight independent FMA chains (a <- a m + c), far more independent work than
// the pipe latency needs, so the FMA pipes are the only limit.  The scalar
// form issues one FFMA per 32 lane-operations, the packed form one FFMA2 per
// 64 (Blackwell's two-wide FP32 FMA), so the packed form is not limited by
// instruction issue.  Nothing of the method is computed here.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sde {
namespace {

constexpr int kChains = 8;   // independent chains per thread
constexpr int kUnroll = 16;  // rounds of the chains per loop iteration

__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, float m, float c, float *sink) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], m, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma2_probe_kernel(int64_t iters, float m, float c, float *sink) {
  float2 a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)j * 1e-3f);
  const float2 M = make_float2(m, m), C = make_float2(c, c);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) a[j] = __ffma2_rn(a[j], M, C);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j].x + a[j].y;
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace sde

extern "C" sde_status sde_fp32_fma_probe(int32_t packed, int64_t iters, int32_t grid, int32_t block,
                                         float *sink_dev, double *flop_host, void *stream) {
  using namespace sde;
  clear_error();
  SDE_CHECK_ARG(packed == 0 || packed == 1, "packed must be 0 or 1");
  SDE_CHECK_ARG(iters >= 1 && iters <= (1ll << 40), "iters must be in [1, 2^40]");
  SDE_CHECK_ARG(grid >= 1 && grid <= (1 << 20), "grid must be in [1, 2^20]");
  SDE_CHECK_ARG(block >= 32 && block <= 256 && block % 32 == 0, "block must be a multiple of 32 in [32, 256]");
  SDE_CHECK_ARG(sink_dev != nullptr, "sink_dev is NULL");
  const double lanes = packed ? 2.0 : 1.0;
  if (flop_host) *flop_host = 2.0 * lanes * kChains * kUnroll * (double)iters * (double)grid * (double)block;
  cudaStream_t s = (cudaStream_t)stream;
  // m and c keep every chain bounded (|a| stays below c / (1 - m)) and finite
  if (packed)
    fma2_probe_kernel<<<grid, block, 0, s>>>(iters, 0.999f, 1e-3f, sink_dev);
  else
    fma_probe_kernel<<<grid, block, 0, s>>>(iters, 0.999f, 1e-3f, sink_dev);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}
