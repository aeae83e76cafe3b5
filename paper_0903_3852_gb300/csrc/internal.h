// internal.h -- context layout and launcher declarations shared by the
// library's translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"
#include "philox.cuh"

namespace sde {

// Per-point FP32 constants of Eq. 1, derived on the device from the FP64
// parameters (prepare kernel).
struct JJConsts {
  float gamma;  // friction
  float a;      // drive amplitude
  float f;      // bias
  float dt;     // 2 pi / (omega P)
  float h;      // dt / 2
  float s;      // sqrt(2 gamma D dt): noise increment per unit Gaussian
  int32_t paths;
  int32_t pad;
  int64_t steps;        // S_k
  int64_t wstart;       // S_k - floor(S_k / 2): window = state indices (wstart, S_k]
  int64_t path_offset;  // global index of the point's first path
  double dt64;          // dt in FP64 (observable times)
};

// A work unit: up to 32 * ILP consecutive paths of one point, advanced by one warp.
struct JJUnit {
  int32_t point;
  int32_t path_begin;  // within the point
  int32_t n_paths;     // <= 32 * ILP
  int32_t pad;
};

// Per-unit reduction partial: count, mean and sum of squared deviations of
// the per-path window averages (merged with Chan's pairwise formula).
struct Moments {
  double n, mean, m2;
};

struct JJUnitList {
  int ilp = 0;
  int32_t n_units = 0;
  JJUnit *units = nullptr;          // device, ordered longest-first
  int2 *point_range = nullptr;      // device, [n_points]: unit range of each point
  std::vector<int2> point_range_h;  // host copy
};

struct JJState {
  const float *x_in, *v_in;
  const int32_t *w_in;
  const double *vsum_in;
  float *x_out, *v_out;
  int32_t *w_out;
  double *vsum_out;
};

struct JJLaunchArgs {
  const JJConsts *consts;
  const JJUnit *units;
  const float *drive;  // [P] cos(2 pi k / P)
  int32_t P;
  int32_t unit_begin;  // first unit of this launch
  int32_t unit_end;    // one past the last unit
  uint32_t *queue;     // persistent: work counter (reset to 0 before launch); plain: NULL
  Moments *partials;   // [n_units]
  uint32_t *err;
  JJState st;
  int64_t n_begin, n_end;
  uint64_t seed;
  PhiloxKeys keys;  // round keys of seed
};

// Kernel launchers (josephson.cu).
cudaError_t jj_prepare(const sde_jj_point *points_dev, int n_points, int P, const int64_t *steps_dev,
                       const int64_t *offsets_dev, const int64_t *paths_dev, JJConsts *consts_dev,
                       float *drive_dev, cudaStream_t s);
cudaError_t jj_launch(const JJLaunchArgs &a, int ilp, int block, int grid, cudaStream_t s);
int jj_max_blocks_per_sm(int ilp, int block, int P);
cudaError_t jj_configure();  // once per process, before the first launch (not under capture)
cudaError_t jj_finalize(const JJConsts *consts, const int2 *point_range, int n_points,
                        const Moments *partials, int64_t n_end, sde_obs_row *obs, cudaStream_t s);

// Histograms (histogram.cu).
cudaError_t winding_hist(const int32_t *w, const int64_t *offsets, const int64_t *paths, int n_points,
                         int64_t max_paths, int32_t w_lo, int32_t nbins, unsigned long long *counts,
                         int sm_count, cudaStream_t s);
cudaError_t phase_hist(const float *phi, int64_t n, int32_t nbins, unsigned long long *counts, int sm_count,
                       cudaStream_t s);

cudaError_t philox_fill(const uint32_t *ctr, uint64_t seed, uint32_t *out, int64_t n, cudaStream_t s);
cudaError_t box_muller_fill(const uint32_t *ctr, uint64_t seed, float *z, int64_t n, cudaStream_t s);
cudaError_t box_muller_words(const uint32_t *w, int64_t n, int variant, float *z, cudaStream_t s);

}  // namespace sde
