// josephson_fp64.cu -- Eq. 1 advanced by Alg. 2 in double precision on the
// GPU, the counterpart of the paper's double-precision run of Fig. 2 (its
// FP32 and FP64 ensembles agree to within the statistical error of the
// histogram, Sec. 5).  It exists to measure the FP32 path's error on the GPU
// itself: same noise stream as the FP32 kernels (Philox4x32-10 block n / 4 of
// counter (path, point, tag 1), identical 24-bit uniforms), with the
// Box-Muller transform, the potential force and the drive evaluated in FP64.
//
// One thread per path, one launch per point; the drive cos(2 pi k / P) for
// k = n mod P is tabulated once per block in shared memory (time modulo the
// period, Sec. 5), and positions are plain FP64 values (53 bits hold the
// fractional part to 1e-12 of a period out to 10^4 periods, so no winding
// count is kept).
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "philox.cuh"

namespace sde {
namespace {

struct JJ64Args {
  double gamma, a, f;
  double dt, h, s;  // dt, dt / 2, sqrt(2 gamma D dt)
  int32_t P;
  uint32_t point;   // noise counter word c2
  int64_t n_paths;
  int64_t n_begin, n_end;
  int64_t wstart;   // the window holds state indices (wstart, S]
  const double *x_in, *v_in, *vsum_in;
  double *x_out, *v_out, *vsum_out;
  uint32_t *err;
  PhiloxKeys keys;
};

// Box-Muller in FP64 from the same 24-bit uniforms as the FP32 path.
__device__ __forceinline__ void box_muller64(uint32_t w0, uint32_t w1, double &z0, double &z1) {
  const double u0 = (double)((w0 >> 8) + 1u) * 5.9604644775390625e-8;  // 2^-24
  const double u1 = (double)((w1 >> 8) + 1u) * 5.9604644775390625e-8;
  const double rho = sqrt(-2.0 * log(u0));
  double sn, cs;
  sincospi(2.0 * u1, &sn, &cs);
  z0 = rho * cs;
  z1 = rho * sn;
}

__device__ __forceinline__ double jj_force64(double x, double v, double drive, const JJ64Args &A) {
  return -A.gamma * v - 6.283185307179586477 * cospi(2.0 * x) + A.a * drive + A.f;
}

__global__ void __launch_bounds__(256) jj64_kernel(const JJ64Args A) {
  extern __shared__ double drive_s[];  // [P]
  for (int k = threadIdx.x; k < A.P; k += blockDim.x) drive_s[k] = cospi((double)(2 * k) / (double)A.P);
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.n_paths) return;
  double x = A.x_in[j], v = A.v_in[j];
  double vs = A.vsum_in ? A.vsum_in[j] : 0.0;
  int32_t k = (int32_t)(A.n_begin % A.P);
  double z[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t n = A.n_begin; n < A.n_end; ++n) {
    const int q = (int)(n & 3);
    if (n == A.n_begin || q == 0) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)(n >> 2), (uint32_t)j, A.point, kTagJosephson), A.keys);
      box_muller64(w.x, w.y, z[0], z[1]);
      box_muller64(w.z, w.w, z[2], z[3]);
    }
    const double psi = q == 0 ? z[0] : (q == 1 ? z[1] : (q == 2 ? z[2] : z[3]));
    const double noise = A.s * psi;
    const int32_t k1 = k + 1 == A.P ? 0 : k + 1;
    // Alg. 2: predictor with F(y_n, t_n), corrector with the mean of the two
    // stages; the same Gaussian in both
    const double F1v = jj_force64(x, v, drive_s[k], A);
    const double xt = x + A.dt * v;
    const double vt = v + A.dt * F1v + noise;
    const double F2v = jj_force64(xt, vt, drive_s[k1], A);
    x = x + A.h * (v + vt);
    v = v + A.h * (F1v + F2v) + noise;
    if (n + 1 > A.wstart) vs += v;
    k = k1;
  }
  if (A.err && !(isfinite(x) && isfinite(v))) atomicOr(A.err, kErrNonFinite);
  A.x_out[j] = x;
  A.v_out[j] = v;
  if (A.vsum_out) A.vsum_out[j] = vs;
}

}  // namespace
}  // namespace sde

extern "C" sde_status sde_josephson_run_fp64(const sde_jj_point *point, int32_t steps_per_period,
                                             int64_t n_paths, int64_t total_steps, uint64_t seed,
                                             uint32_t point_index, int64_t n_begin, int64_t n_end,
                                             const double *x_in_dev, const double *v_in_dev,
                                             const double *vsum_in_dev, double *x_out_dev,
                                             double *v_out_dev, double *vsum_out_dev, uint32_t *err_dev,
                                             void *stream) {
  using namespace sde;
  SDE_CHECK_ARG(point != nullptr, "point is NULL");
  SDE_CHECK_ARG(n_paths >= 0 && n_paths < (1ll << 31), "n_paths must be in [0, 2^31)");
  SDE_CHECK_ARG(steps_per_period >= 1 && steps_per_period <= 4096, "steps_per_period must be in [1, 4096]");
  SDE_CHECK_ARG(total_steps >= 0 && total_steps <= (1ll << 33), "total_steps out of range");
  SDE_CHECK_ARG(n_begin >= 0 && n_end >= n_begin && n_end <= (1ll << 33), "need 0 <= n_begin <= n_end");
  SDE_CHECK_ARG(isfinite(point->gamma) && isfinite(point->a) && isfinite(point->omega) && isfinite(point->f) &&
                    isfinite(point->D),
                "point parameters must be finite");
  SDE_CHECK_ARG(point->omega > 0.0 && point->gamma > 0.0 && point->D >= 0.0,
                "need omega > 0, gamma > 0, D >= 0");
  if (n_paths == 0) return SDE_OK;
  SDE_CHECK_ARG(x_in_dev && v_in_dev && x_out_dev && v_out_dev, "x/v buffers must be non-NULL");
  JJ64Args a{};
  a.gamma = point->gamma;
  a.a = point->a;
  a.f = point->f;
  a.dt = 2.0 * 3.14159265358979323846 / (point->omega * (double)steps_per_period);
  a.h = 0.5 * a.dt;
  a.s = sqrt(2.0 * point->gamma * point->D * a.dt);
  a.P = steps_per_period;
  a.point = point_index;
  a.n_paths = n_paths;
  a.n_begin = n_begin;
  a.n_end = n_end < total_steps ? n_end : total_steps;  // a point stops at its S
  if (a.n_end < a.n_begin) a.n_end = a.n_begin;
  a.wstart = total_steps - total_steps / 2;
  a.x_in = x_in_dev;
  a.v_in = v_in_dev;
  a.vsum_in = vsum_in_dev;
  a.x_out = x_out_dev;
  a.v_out = v_out_dev;
  a.vsum_out = vsum_out_dev;
  a.err = err_dev;
  a.keys = philox_round_keys(seed);
  const int block = 256;
  const size_t smem = sizeof(double) * (size_t)steps_per_period;
  const unsigned grid = (unsigned)((n_paths + block - 1) / block);
  jj64_kernel<<<grid, block, smem, (cudaStream_t)stream>>>(a);
  SDE_CUDA_TRY(cudaGetLastError());
  return SDE_OK;
}
