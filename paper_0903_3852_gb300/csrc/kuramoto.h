// kuramoto.h -- Kuramoto (Eq. 2) part of the library: context and entry
// points used by abi.cu.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace sde {

struct KuramotoCtx;

// Host-side checks of a Kuramoto configuration (no CUDA call); kuramoto_create
// runs them first as well.
sde_status kuramoto_validate(const sde_config *cfg);
sde_status kuramoto_create(const sde_config *cfg, int sm_count, uint32_t *err, KuramotoCtx **out);
// Advance and reduce; (re)allocates the observables buffer *obs if it has
// fewer than the run's sample rows.  ev0/ev1 bracket the dominant kernels.
sde_status kuramoto_run(KuramotoCtx *k, const sde_run_desc *r, cudaStream_t s, cudaEvent_t ev0,
                        cudaEvent_t ev1, sde_obs_row *obs_in, sde_obs_row **obs,
                        int64_t *max_rows, int64_t *rows);
sde_status kuramoto_set_coupling(KuramotoCtx *k, const float *K_dev, cudaStream_t s);
// out[r][i] = sum_j K_ij sin(phi_j - phi_i) through the model's coupling path.
sde_status kuramoto_coupling(KuramotoCtx *k, const float *phi_dev, float *out_dev, cudaStream_t s);
void kuramoto_tuning(const KuramotoCtx *k, int32_t *block, int32_t *per_thread, int32_t *cluster);
// Mean and total device time of the dominant kernel's launches in the last
// run, when they were timed per launch; false if they were not.
bool kuramoto_kernel_stats(KuramotoCtx *k, float *mean_ms, float *total_ms, int64_t *launches);
void kuramoto_destroy(KuramotoCtx *k);
// Limit (ns) of the bounded device waits of the context's later launches.
void kuramoto_set_wait_limit(KuramotoCtx *k, uint64_t ns);

}  // namespace sde
