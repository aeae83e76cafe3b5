// kuramoto_internal.h -- Kuramoto context and kernel arguments shared by
// kuramoto.cu and kuramoto_general.cu.  Not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace sde {

struct KuramotoCtx {
  int model = 0;
  int64_t N = 0, R = 0;
  double K = 0.0, D = 0.0, dt = 0.0;
  int M = 0;
  uint64_t seed = 0;
  int sm_count = 0;
  uint32_t *err = nullptr;
  uint64_t wait_ns = 1000000000ull;  // limit of the kernels' bounded device waits
  uint32_t flags = 0;
  int block = 0, opt = 0;
  int cs = 1;  // mean field: CTAs per replica (thread-block cluster size); 0 = grid-wide form
  bool mf_async = false;  // cluster exchange by asynchronous remote stores + mbarrier
  // grid-wide mean field: per-replica partial sums, totals and block counters
  int mfg_blocks = 0;             // blocks per replica, the largest of mfg_grid
  int mfg_grid[4] = {0, 0, 0, 0}; // blocks per replica: predictor, corrector, sums, predictor drawing noise
  float2 *mfg_partials = nullptr; // [R][mfg_blocks]
  double *mfg_tot = nullptr;      // [R][4]: S, C of theta_n, then S, C of theta~_n
  uint32_t *mfg_count = nullptr;  // [R]
  // phases as fixed-point turns, [R][N]
  uint32_t *theta = nullptr;
  uint32_t *theta_t = nullptr;  // predictor phases (pairwise, general, grid-wide mean field)
  float *g1 = nullptr;          // first-stage coupling sums (pairwise, general); grid-wide
                                // mean field: the first-stage part of the step increment
  double *r_scratch = nullptr;  // r samples when the caller passes none
  int64_t r_scratch_rows = 0;
  // general coupling
  float *Kf32 = nullptr;          // [N][N] FP32 copy (CUDA-core baseline)
  __nv_bfloat16 *Kbf16 = nullptr; // [N][N] BF16 copy (tensor-core path)
  __nv_bfloat16 *Bt = nullptr;    // [2R][N] sin / cos rows (BF16 operand)
  float *Bt32 = nullptr;          // [2R][N] sin / cos rows (FP32 operand)
  float *P = nullptr;             // [2R][N] GEMM output (transposed)
  float *psi4 = nullptr;          // general: [2][4][R][N] Gaussians of two 4-step Philox blocks; grid-wide mean field: [3][R][N]
  bool have_K = false;
  void *gemm_plan = nullptr;
  // per-launch timing of the dominant kernel (SDE_FLAG_TIME_KERNELS)
  std::vector<cudaEvent_t> kev;
  int64_t kev_used = 0;      // event pairs recorded
  int64_t kev_launches = 0;  // launches those pairs bracket
};

// Record the start / end of one launch of the dominant kernel when the
// context times kernels; no-ops otherwise.
cudaError_t ktime_begin(KuramotoCtx *k, cudaStream_t s);
cudaError_t ktime_end(KuramotoCtx *k, cudaStream_t s, int64_t launches = 1);

// Arguments of the mean-field kernel.
struct KurArgs {
  const uint32_t *theta_in;
  uint32_t *theta_out;
  const float *omega;
  double *r_out;  // [samples][R]
  int64_t N, R;
  int64_t n_begin, n_end;
  int32_t M;
  float wscale;  // dt / (2 pi): radians per unit time -> turns per step
  float kc;      // (K / N) dt / (2 pi)
  float kh;      // kc / 2
  float sc;      // sqrt(2 D dt) / (2 pi)
  uint64_t seed;
  uint32_t *err;
  uint64_t wait_ns;  // limit of each bounded mbarrier wait (asynchronous exchange)
};

// Arguments of one pairwise stage launch.
struct KurPairArgs {
  uint32_t *theta;
  uint32_t *theta_t;
  float *g1;
  const float *omega;
  int64_t N;
  int64_t n;
  float wscale, kc, kh, sc;
  uint64_t seed;
};

cudaError_t kur_order_launch(const uint32_t *theta, int64_t N, int64_t R, double *r_out, cudaStream_t s);

sde_status kuramoto_general_alloc(KuramotoCtx *k);
void kuramoto_general_free(KuramotoCtx *k);
sde_status kuramoto_general_run(KuramotoCtx *k, const sde_run_desc *r, cudaStream_t s, double *rbuf);
sde_status kuramoto_general_coupling(KuramotoCtx *k, float *out, cudaStream_t s);

}  // namespace sde
