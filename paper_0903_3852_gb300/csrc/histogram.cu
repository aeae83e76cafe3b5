// histogram.cu -- coarse-grained densities of the ensembles (the histograms
// of Fig. 2 and Fig. 4).
//
// Fig. 2 bins the particle position with bins exactly one potential period
// wide (Sec. 5), i.e. by the integer part of x: with the state kept as
// x in [0, 1) plus a winding count w, the bin is w itself, exact integer
// arithmetic.  Fig. 4 shows the density P(x; t) of the Kuramoto phases
// modulo 2 pi.  Counts are integers accumulated with shared-memory and then
// global atomics, so results do not depend on thread order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sde {
namespace {

// One block per (point, chunk of paths): counts[point][0] = below w_lo,
// counts[point][1 + b] = w_lo + b, counts[point][nbins + 1] = above.
__global__ void winding_hist_kernel(const int32_t *w, const int64_t *offsets, const int64_t *paths,
                                    int32_t w_lo, int32_t nbins, unsigned long long *counts) {
  extern __shared__ unsigned int h[];
  const int p = blockIdx.y;
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  const int64_t n = paths[p], off = offsets[p];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rel = (int64_t)w[off + j] - (int64_t)w_lo;
    const int bin = rel < 0 ? 0 : (rel >= nbins ? nbins + 1 : (int)rel + 1);
    atomicAdd(&h[bin], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins + 2; b += blockDim.x)
    if (h[b]) atomicAdd(&counts[(int64_t)p * (nbins + 2) + b], (unsigned long long)h[b]);
}

// Phases in radians, expected in [0, 2 pi): bin = floor(phi * (nbins / 2 pi)) in
// FP32, clamped to [0, nbins - 1].
__global__ void phase_hist_kernel(const float *phi, int64_t n, int32_t nbins, float scale,
                                  unsigned long long *counts) {
  extern __shared__ unsigned int h[];
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0u;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int bin = (int)floorf(phi[i] * scale);
    bin = bin < 0 ? 0 : (bin >= nbins ? nbins - 1 : bin);
    atomicAdd(&h[bin], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x)
    if (h[b]) atomicAdd(&counts[b], (unsigned long long)h[b]);
}

}  // namespace

cudaError_t winding_hist(const int32_t *w, const int64_t *offsets, const int64_t *paths, int n_points,
                         int64_t max_paths, int32_t w_lo, int32_t nbins, unsigned long long *counts,
                         int sm_count, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)n_points * (nbins + 2), s);
  if (e != cudaSuccess || max_paths == 0) return e;
  const int64_t chunks = (max_paths + 255) / 256;
  const int gx = (int)(chunks < 64 ? chunks : 64);
  winding_hist_kernel<<<dim3(gx, n_points), 256, sizeof(unsigned int) * (nbins + 2), s>>>(w, offsets, paths, w_lo,
                                                                                         nbins, counts);
  (void)sm_count;
  return cudaGetLastError();
}

cudaError_t phase_hist(const float *phi, int64_t n, int32_t nbins, unsigned long long *counts, int sm_count,
                       cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * (size_t)nbins, s);
  if (e != cudaSuccess || n == 0) return e;
  const int64_t blocks = (n + 255) / 256;
  const int g = (int)(blocks < (int64_t)sm_count * 8 ? blocks : (int64_t)sm_count * 8);
  const float scale = (float)((double)nbins / 6.28318530717958647692);
  phase_hist_kernel<<<g, 256, sizeof(unsigned int) * nbins, s>>>(phi, n, nbins, scale, counts);
  return cudaGetLastError();
}

}  // namespace sde
