/*
 * sde.h -- C ABI of the GB300 ensemble-SDE library (libsde_gb300.so).
 *
 * Januszewski & Kostur, "Accelerating numerical solution of stochastic
 * differential equations with CUDA" (arXiv:0903.3852).  The library
 * integrates many independent realisations of
 *   Eq. 1 (Sec. 3)  x'' + gamma x' = -2 pi cos(2 pi x) + a cos(omega t) + f
 *                                   + sqrt(2 gamma D) xi(t)
 *   Eq. 2 (Sec. 3)  x_i' = omega_i + sum_j K_ij sin(x_j - x_i) + sqrt(2 D) xi_i(t)
 *                   (gamma = 1)
 * with the second-order stochastic Runge-Kutta step of Alg. 2 (Heun form,
 * the same Gaussian in both stages), Gaussian noise from Philox4x32-10
 * counters through Box-Muller (Sec. 4.1), and FP64 on-device ensemble
 * reductions (Sec. 4.1, ensemble averages; Sec. 5, <<v>>).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *    library never frees them.  *_host pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every kernel goes on that stream; no entry point
 *    synchronises the device except sde_observables and sde_last_kernel_ms.
 *  - Every entry point returns an sde_status; on failure the thread-local
 *    message from sde_last_error() says why.  No exception crosses the ABI.
 *  - Asynchronous device faults found by the kernels (non-finite state, a
 *    bounded wait that expired) are latched in the context and returned by
 *    the next sde_observables call.
 */
#ifndef SDE_GB300_H_
#define SDE_GB300_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sde_status {
  SDE_OK = 0,
  SDE_ERR_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
  SDE_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has it)   */
  SDE_ERR_NO_MEMORY = 3,   /* device or host allocation failed             */
  SDE_ERR_TIMEOUT = 4,     /* a bounded device wait expired                */
  SDE_ERR_UNSUPPORTED = 5, /* valid request this build does not implement  */
  SDE_ERR_NUMERIC = 6      /* a kernel produced a non-finite state         */
} sde_status;

typedef enum sde_model {
  SDE_JOSEPHSON = 0,          /* Eq. 1, per-path kernels (Alg. 1)              */
  SDE_KURAMOTO_MEANFIELD = 1, /* Eq. 2, K_ij = K/N, mean-field sums (Eq. 3)     */
  SDE_KURAMOTO_PAIRWISE = 2,  /* Eq. 2, K_ij = K/N, direct all-pairs sum (Alg. 3) */
  SDE_KURAMOTO_GENERAL = 3,   /* Eq. 2, matrix K_ij: BF16 tensor-core GEMM      */
  SDE_KURAMOTO_GENERAL_FP32 = 4 /* Eq. 2, matrix K_ij: FP32 CUDA-core baseline  */
} sde_model;

/* Launch schedules.  Josephson: PERSISTENT or PLAIN.  Kuramoto mean field:
   PERSISTENT picks the form (a replica per CTA or thread-block cluster when
   n_osc <= 8192, autotuned against the grid-wide form when replicas are
   few; the grid-wide form above 8192), GRID forces the grid-wide form.  The
   other Kuramoto models take PERSISTENT (0). */
typedef enum sde_schedule {
  SDE_SCHED_PERSISTENT = 0, /* all points in one persistent launch with a work
                               queue ordered longest-first, graph-captured   */
  SDE_SCHED_PLAIN = 1,      /* one launch per point, one thread per path
                               (the per-path kernel of Alg. 1)               */
  SDE_SCHED_GRID = 2        /* Kuramoto mean field (Eq. 3) with each replica
                               spread over the whole grid: two launches per
                               step, sums reduced by the last block of each
                               (the form for the 2^24 oscillators of Fig. 4) */
} sde_schedule;

/* Flags for sde_config.flags. */
#define SDE_FLAG_NO_GRAPH 1u     /* launch kernels directly instead of replaying a graph */
#define SDE_FLAG_TIME_KERNELS 2u /* Kuramoto pairwise / general: CUDA events around every
                                    launch of the dominant kernel (stage / GEMM); for the
                                    general coupling around the GEMMs of every 8th step only,
                                    or with SDE_FLAG_FUSED around the whole run of back-to-back
                                    GEMMs (events between GEMMs keep the next one's prologue
                                    from overlapping the previous one's end) */
#define SDE_FLAG_FUSED 4u        /* general coupling, tensor-core form: run the SRK2
                                    sub-steps in the GEMM epilogue instead of as
                                    separate kernels (same results bit for bit) */
#define SDE_FLAG_ASYNC_EXCHANGE 16u /* Kuramoto mean field in clusters: exchange the partial sums
                                        by asynchronous remote stores that complete on the
                                        receiving CTA's mbarrier, instead of a cluster barrier
                                        (the autotuner tries both forms when unset) */
#define SDE_FLAG_GEMM_SINGLE_CTA 32u /* general coupling, tensor-core form: whole tiles, one CTA
                                        per 128 x 256 tile of the GEMM (tcgen05 cta_group::1),
                                        instead of the CTA-pair GEMM (a 256 x 256 tile per
                                        cluster of two CTAs, cta_group::2) that whole tiles use by
                                        default where n_osc % 256 == 0 and n_replicas % 128 == 0
                                        (same results bit for bit) */
#define SDE_FLAG_GEMM_STREAM_K 64u /* general coupling, tensor-core form (n_replicas % 128 == 0):
                                      split the K range of all 128 x 256 tiles evenly over as many
                                      CTAs as can be resident (stream-K); each tile's first CTA
                                      adds the others' FP32 partial sums (equal to the whole-tile
                                      GEMM up to the rounding of those sums, deterministic on a
                                      given GPU).  A split K slice costs about 1.4 times a
                                      whole-tile one, so this pays only where whole tiles fill
                                      few SMs and K is long (N = 8192 with 128 replicas: 9 %
                                      faster); not at N = 8192 with 256 replicas */
#define SDE_FLAG_EULER 8u        /* Euler-Maruyama instead of SRK2 (Alg. 2): the
                                    first-order scheme of PROG2 (Sec. 4.2).
                                    Josephson: every schedule, same kernels with
                                    the one-stage step.  Kuramoto pairwise: PROG2's
                                    two kernels per step, UpdateRHS (the tiled
                                    all-pairs sum of Alg. 3, stored) then
                                    AdvanceSystem (phi += dt drift + noise).  Other
                                    Kuramoto models: SDE_ERR_UNSUPPORTED */

/* One parameter point of Eq. 1. */
typedef struct sde_jj_point {
  double gamma; /* friction, > 0                          */
  double a;     /* drive amplitude                        */
  double omega; /* drive angular frequency, > 0           */
  double f;     /* constant bias                          */
  double D;     /* noise intensity k_B T, >= 0            */
} sde_jj_point;

typedef struct sde_config {
  int32_t model;    /* sde_model                                             */
  int32_t schedule; /* sde_schedule                                          */
  uint64_t seed;    /* Philox key: (seed & 0xffffffff, seed >> 32)           */

  /* ---- Josephson (Eq. 1) -------------------------------------------- */
  int32_t n_points;         /* >= 1                                          */
  int32_t steps_per_period; /* P in [1, 4096]: dt_k = 2 pi / (omega_k P); the
                               drive phase is kept as the integer n mod P
                               (time modulo the period, Sec. 5)             */
  const sde_jj_point *points; /* host, n_points entries; copied at create  */
  const int64_t *paths;       /* host, paths per point, each in [0, 2^31)   */
  const int64_t *steps;       /* host, total steps S_k per point, [0, 2^33];
                                 <v> averages v over the last floor(S_k/2)
                                 states                                     */

  /* ---- Kuramoto (Eq. 2) --------------------------------------------- */
  int64_t n_osc;        /* N oscillators per replica                        */
  int64_t n_replicas;   /* independent replicas                             */
  double K;             /* uniform models: K_ij = K / N                     */
  double D;             /* noise intensity                                  */
  double dt;            /* time step                                        */
  int32_t sample_every; /* M: r(t) is sampled every M steps (M = 100 in the
                           paper, Sec. 4.1); 0 = no samples                  */

  /* ---- tuning --------------------------------------------------------- */
  int32_t block_threads;    /* threads per block; 0 = autotune               */
  int32_t paths_per_thread; /* Josephson paths per thread: 1, 2 or 4 (2 and 4 advance
                               pairs of paths with packed FP32x2 instructions),
                               or 11 / 12 / 14 for 1 / 2 / 4 with fewer
                               registers (64 / 64 / 96); 0 = autotune          */
  uint32_t flags;           /* SDE_FLAG_*                                     */
  int32_t cluster_ctas;     /* Kuramoto mean field: CTAs per replica (1, 2, 4 or
                               8, a thread-block cluster above 1); 0 = autotune
                               together with block_threads                     */
} sde_config;

/*
 * Arguments of one sde_run_ensemble call.  The state arrays are
 * caller-owned device buffers; *_in and *_out may alias (in-place run).
 *
 * Josephson layout: structure of arrays, point-major: the paths of point 0,
 * then those of point 1, ... (total = sum of paths).  Position is stored as
 * a fractional part x in [0, 1) plus an int32 winding count w (x_abs = w +
 * x); the kernels wrap any x_in on load.  vsum holds the running sum of v
 * over the averaging window (FP64).  w_in and vsum_in may be NULL (zeros).
 *
 * Kuramoto layout: replica-major [replica][oscillator], phases in radians;
 * phi_out is wrapped to [0, 2 pi).  omega is [replica][oscillator].
 */
typedef struct sde_run_desc {
  int64_t n_begin; /* first step index (the noise counter)                  */
  int64_t n_end;   /* one past the last step; Josephson points stop at S_k  */
  /* Josephson */
  const float *x_in_dev;
  const float *v_in_dev;
  const int32_t *w_in_dev;
  const double *vsum_in_dev;
  float *x_out_dev;
  float *v_out_dev;
  int32_t *w_out_dev;
  double *vsum_out_dev;
  /* Kuramoto */
  const float *phi_in_dev;
  float *phi_out_dev;
  const float *omega_dev;
  double *r_out_dev; /* [n_samples][n_replicas] or NULL; n_samples =
                        ceil((n_end - n_begin) / M) + 1, the last at n_end  */
} sde_run_desc;

/* One row of observables (FP64). */
typedef struct sde_obs_row {
  double mean;  /* Josephson: ensemble mean of the per-path time average of v
                   over the window; Kuramoto: mean over replicas of r(t)     */
  double var;   /* unbiased variance of the same per-path / per-replica values */
  double se;    /* standard error sqrt(var / count)                         */
  double count; /* number of paths (replicas) in the row                    */
  double t;     /* Josephson: time at the end of the window; Kuramoto: t_n  */
} sde_obs_row;

typedef struct sde_ctx sde_ctx; /* opaque, library-owned */

/*
 * Validate cfg, copy the parameter tables to the device, allocate the
 * library workspace (work list, reduction partials, observables) and, if
 * block_threads or paths_per_thread is 0, autotune the launch shape by
 * timing short runs of each candidate on the current device.  The context
 * is bound to the current CUDA device.
 * Errors: SDE_ERR_INVALID_ARG (bad sizes or parameters) and
 * SDE_ERR_UNSUPPORTED (a flag the model does not implement) are found on the
 * host before any CUDA call, so they are reported the same with or without a
 * GPU; then SDE_ERR_NO_MEMORY, SDE_ERR_CUDA.  On error *out is NULL.
 */
sde_status sde_create(const sde_config *cfg, sde_ctx **out);

/*
 * Advance the ensemble from step run->n_begin to run->n_end on `stream`
 * (Alg. 1: load state, loop over steps, store state) and reduce the
 * observables on the device (FP64).  Josephson points whose S_k <= n_begin
 * are left unchanged.  Asynchronous; the state buffers must stay valid
 * until the stream reaches the end of the call's work.
 * Errors: SDE_ERR_INVALID_ARG (NULL required pointer, n_end < n_begin),
 * SDE_ERR_CUDA (launch failure).
 */
sde_status sde_run_ensemble(sde_ctx *ctx, const sde_run_desc *run, void *stream);

/*
 * Synchronise the stream of the last run and copy the observables of that
 * run to rows_host: one row per point (Josephson) or per sample time
 * (Kuramoto).  *n_rows receives the row count; if capacity is smaller, only
 * the first `capacity` rows are copied.  Returns the latched device status
 * (SDE_ERR_TIMEOUT before SDE_ERR_NUMERIC) if a kernel reported one since the
 * last call; a reported status is cleared, so later runs start clean.
 */
sde_status sde_observables(sde_ctx *ctx, sde_obs_row *rows_host, int64_t capacity,
                           int64_t *n_rows);

/* Free the context and its workspace.  NULL-safe.  Synchronises the device. */
void sde_destroy(sde_ctx *ctx);

/*
 * Failure detection (the paper has no counterpart).  Kernels that wait on
 * other threads through mbarriers -- the tensor-core GEMM of
 * SDE_KURAMOTO_GENERAL (its TMA producer and MMA issuer) and the Kuramoto
 * mean field with SDE_FLAG_ASYNC_EXCHANGE -- bound every such wait by a
 * limit of the GPU's nanosecond timer.  When one expires the kernel stops
 * issuing work, drains what it has issued (with waits of at most one second,
 * whatever the limit), latches SDE_ERR_TIMEOUT for the next sde_observables
 * and returns; the context stays usable.  This sets the limit for the
 * context's later launches: ns = 0 restores the default of one second.  A
 * small limit makes the waits expire on purpose, for tests of that path.
 * Josephson contexts have no such waits (the call succeeds and changes
 * nothing).  Errors: SDE_ERR_INVALID_ARG (NULL ctx).
 */
sde_status sde_set_wait_limit(sde_ctx *ctx, uint64_t ns);

/*
 * Allocation-failure injection for tests (the paper has no counterpart):
 * during the next sde_create or sde_mlp_create call, its nth allocation
 * (1 = the host context of sde_create, then the device buffers in the order
 * the call makes them, its autotuning scratch included) fails as if memory
 * had run out, so the call returns SDE_ERR_NO_MEMORY, frees what it had
 * allocated and leaves *out NULL.  Each create call disarms the injection
 * when it returns; nth <= 0 disarms it now.  Process-wide.
 */
void sde_debug_fail_allocation(int32_t nth);

/* Message of the last failed call on this thread ("" if none). */
const char *sde_last_error(void);

/* Launch shape chosen at create (after autotuning): threads per block, paths
   (Josephson; values 11 and 12 mean 1 and 2 with registers capped at 64) or
   oscillators (Kuramoto) per thread, and CTAs per replica (the thread-block
   cluster of the mean-field kernel; 0 for the grid-wide mean field, whose
   per-thread count is then the oscillators each thread strides over; for the
   general coupling's tensor-core GEMM, the CTAs per tile: 2 for the CTA-pair
   GEMM, whose per-thread value is then the D columns of a tile, 0 for the
   stream-K split (SDE_FLAG_GEMM_STREAM_K), whose per-thread value is then
   the CTAs of the split grid;
   1 otherwise).  Any pointer may be NULL. */
sde_status sde_get_tuning(const sde_ctx *ctx, int32_t *block_threads, int32_t *per_thread,
                          int32_t *cluster_ctas);

/*
 * Device time of the dominant kernel of the last run, from CUDA events
 * recorded on the run's stream around it: the persistent or per-point
 * Josephson launches, the mean-field kernel, or -- with
 * SDE_FLAG_TIME_KERNELS -- each pairwise stage launch, each GEMM launch of
 * every 8th step, or (SDE_FLAG_FUSED) the run's GEMMs as one block (mean_ms
 * per timed launch, total_ms summed over the timed events, launches = the
 * launches they bracket).  Without that flag the
 * Kuramoto loop is bracketed as one launch.  Synchronises that stream.
 * sde_last_kernel_ms returns mean_ms.
 */
sde_status sde_last_kernel_stats(sde_ctx *ctx, float *mean_ms, float *total_ms, int64_t *launches);
sde_status sde_last_kernel_ms(sde_ctx *ctx, float *ms);

/*
 * Load the coupling matrix of the general Kuramoto models (Eq. 2, K_ij):
 * K_dev is N x N FP32, row-major, row i = the oscillator that receives
 * sum_j K_ij sin(x_j - x_i).  SDE_KURAMOTO_GENERAL keeps a BF16 copy (the
 * tensor-core operand), SDE_KURAMOTO_GENERAL_FP32 an FP32 copy; K_dev may be
 * freed once the stream has passed this call.  Must precede sde_run_ensemble.
 * Errors: SDE_ERR_INVALID_ARG (not a general model, NULL K).
 */
sde_status sde_set_coupling(sde_ctx *ctx, const float *K_dev, void *stream);

/*
 * Coupling sums of Eq. 2 for every replica through the context's coupling
 * path: out_dev[r][i] = sum_j K_ij sin(phi_j - phi_i) (uniform models:
 * K_ij = K/N; mean-field form of Eq. 3 evaluated pairwise; general models:
 * the GEMM form, BF16 or FP32).  phi_dev, out_dev: [n_replicas][n_osc] FP32.
 */
sde_status sde_kuramoto_coupling(sde_ctx *ctx, const float *phi_dev, float *out_dev, void *stream);

/*
 * Coarse-grained position histogram of a Josephson ensemble (Fig. 2, Sec. 5:
 * bins exactly one potential period wide): for every point k, counts of the
 * winding count w (the integer part of the position) of its paths, from the
 * w array of a run (w_out_dev).  counts_dev[k][0] counts w < w_lo,
 * counts_dev[k][1 + b] counts w = w_lo + b (b < nbins) and
 * counts_dev[k][nbins + 1] counts w >= w_lo + nbins.  counts_dev: device,
 * n_points x (nbins + 2) unsigned 64-bit, overwritten.  nbins in [1, 8192].
 */
sde_status sde_position_histogram(sde_ctx *ctx, const int32_t *w_dev, int32_t w_lo, int32_t nbins,
                                  unsigned long long *counts_dev, void *stream);

/*
 * Phase density of Kuramoto ensembles (Fig. 4, P(x; t)): counts of n phases
 * phi_dev (radians, as returned by a run: [0, 2 pi)) in nbins equal bins;
 * bin = floor(phi * (float)(nbins / 2 pi)) in FP32, clamped to [0, nbins-1].
 * counts_dev: device, nbins unsigned 64-bit, overwritten.
 */
sde_status sde_phase_histogram(const float *phi_dev, int64_t n, int32_t nbins, unsigned long long *counts_dev,
                               void *stream);

/*
 * Philox4x32-10 (Salmon et al., SC'11; replaces the xorshift generator of
 * Sec. 4.1): out_dev[4i..4i+3] = Philox(counter ctr_dev[4i..4i+3], key =
 * (seed low word, seed high word)).  n counters, n >= 0, device arrays.
 */
sde_status sde_philox4x32_10(const uint32_t *ctr_dev, uint64_t seed, uint32_t *out_dev,
                             int64_t n, void *stream);

/*
 * Box-Muller Gaussians (Sec. 4.1) as the integrators draw them: for each of
 * the n counters, z_dev[4i..4i+3] = (z0, z1) from words (0, 1) and (z2, z3)
 * from words (2, 3), with u = ((w >> 8) + 1) 2^-24, z0 = sqrt(-2 ln u0)
 * cos(2 pi u1), z1 = sqrt(-2 ln u0) sin(2 pi u1), in FP32.
 */
sde_status sde_box_muller(const uint32_t *ctr_dev, uint64_t seed, float *z_dev, int64_t n,
                          void *stream);

/*
 * The Box-Muller transform (Sec. 4.1) of given 32-bit word pairs:
 * w_dev[2i], w_dev[2i+1] -> z_dev[2i], z_dev[2i+1] (device arrays, 8-byte
 * aligned), with the uniforms of sde_box_muller.  variant 0: the transform
 * the Kuramoto and surrogate kernels use (accurate logf, sin/cos of the
 * fixed-point angle); variant 1: the Josephson kernels' (angle from a
 * 1024-entry table plus angle addition; ln u0 from the hardware base-2
 * logarithm: the radius is within ~5e-4 absolute, and within ~1e-7
 * relative for u0 well below 1).  For exhaustive checks of both.
 */
sde_status sde_box_muller_words(const uint32_t *w_dev, int64_t n_pairs, int32_t variant, float *z_dev,
                                void *stream);

/*
 * Allocation-free run of one Josephson parameter point.  The paper has no
 * counterpart: this is an interface for callers that must not allocate
 * device memory -- code running inside another framework's memory pool or
 * arena, which forbids allocations it does not manage; code invoked while a
 * host program captures the stream into a CUDA graph, where cudaMalloc is
 * not allowed; and hosts that reserve all device memory at start-up.
 *
 * It computes what sde_create + sde_run_ensemble + the observables would
 * for a single point with the plain schedule (one thread per path, warps of
 * 32 paths): same state layout and meaning as sde_run_desc, one
 * sde_obs_row written to obs_dev (device).  It calls no cudaMalloc,
 * cudaFree or allocating library routine.  Its only scratch, one reduction
 * partial per 32 paths, is a fixed array of SDE_NOALLOC_MAX_PATHS / 32
 * entries (768 KiB) in the library's static device memory, held by every
 * GPU that loads the library until the process exits.
 *
 *  - n_paths above SDE_NOALLOC_MAX_PATHS returns SDE_ERR_INVALID_ARG.
 *  - The first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress, with that device current); make the first call
 *    on a device before any stream capture begins.  The address is kept for
 *    the life of the process, so resetting the device (cudaDeviceReset, or
 *    anything else that destroys its primary context) between calls is not
 *    supported.
 *  - All calls on a device share the array.  Calls that can overlap on the
 *    GPU (different streams without ordering, or host threads) race on it
 *    and must be serialised by the caller.  Each call writes every entry it
 *    reads, so leftovers from earlier calls do no harm.
 *  - Non-finite states are not latched; they appear in the outputs.
 */
#define SDE_NOALLOC_MAX_PATHS (1 << 20)

sde_status sde_josephson_run_noalloc(const sde_jj_point *point_host, int32_t steps_per_period,
                                     int64_t n_paths, int64_t total_steps, uint64_t seed,
                                     int64_t n_begin, int64_t n_end, const float *x_in_dev,
                                     const float *v_in_dev, const int32_t *w_in_dev,
                                     const double *vsum_in_dev, float *x_out_dev, float *v_out_dev,
                                     int32_t *w_out_dev, double *vsum_out_dev, sde_obs_row *obs_dev,
                                     void *stream);

/*
 * Double-precision run of one Eq. 1 parameter point: Alg. 2 with every
 * operation in FP64, the counterpart of the paper's double-precision GPU
 * run of Fig. 2 (Sec. 5 compares its histograms with the FP32 run's).  The
 * noise is the FP32 path's stream -- Philox4x32-10 block n / 4 of counter
 * (path, point_index, tag 1), the same 24-bit uniforms -- with Box-Muller in
 * FP64, so an FP32 and an FP64 run of the same point draw the same
 * Gaussians up to FP32 rounding.
 *
 *  - x is the absolute position in units of the potential period (no
 *    winding split), v the velocity; [n_paths] FP64 device arrays, caller-
 *    owned; *_in and *_out may alias.  vsum_in / vsum_out (nullable) carry
 *    the running sum of v over the window (S - floor(S/2), S] of state
 *    indices, S = total_steps; the run stops at S.
 *  - Steps [n_begin, n_end) are taken; splitting a run at any step gives
 *    the same result bit for bit.
 *  - err_dev (nullable, device) gets bit 1 ORed in when a path ends
 *    non-finite.  Asynchronous on `stream`; no allocation.
 *  - Invalid sizes or parameters return SDE_ERR_INVALID_ARG before any
 *    CUDA call.
 */
sde_status sde_josephson_run_fp64(const sde_jj_point *point_host, int32_t steps_per_period,
                                  int64_t n_paths, int64_t total_steps, uint64_t seed,
                                  uint32_t point_index, int64_t n_begin, int64_t n_end,
                                  const double *x_in_dev, const double *v_in_dev,
                                  const double *vsum_in_dev, double *x_out_dev, double *v_out_dev,
                                  double *vsum_out_dev, uint32_t *err_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Learned surrogate of <<v>> (not in the paper).                          */
/*                                                                         */
/* An ensemble of n_members multilayer perceptrons n_in -> hidden (x      */
/* n_hidden layers, SiLU) -> 1, mapping the parameters of Eq. 1 to the     */
/* time-averaged velocity <<v>> of Sec. 5.  FP32 master weights and Adam   */
/* moments; every GEMM takes BF16 operands (weights and activations        */
/* rounded from FP32) and accumulates in FP32.  The ensemble spread is the  */
/* network's own error estimate.  Parameters of one member are stored      */
/* flat as [W1, b1, W2, b2, ..., W_L, b_L], W_l row-major (out, in).       */
/* ---------------------------------------------------------------------- */
typedef struct sde_mlp sde_mlp; /* opaque */

typedef struct sde_mlp_config {
  int32_t n_in;      /* inputs, 1..8 (the surrogate uses 5)                 */
  int32_t hidden;    /* width of every hidden layer, multiple of 64, <= 1024 */
  int32_t n_hidden;  /* hidden layers, 1..8                                 */
  int32_t n_members; /* ensemble size, 1..16                                */
  int64_t max_batch; /* largest batch of any call, >= 1                     */
  float lr, beta1, beta2, eps; /* Adam (Kingma & Ba, Algorithm 1)          */
  uint64_t seed;     /* initial weights: U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from Philox */
  /* feature map of sde_mlp_features: feature k = 2 (p_k - lo_k) / (hi_k - lo_k) - 1
     for p = (a, omega, f, gamma, log10 D) */
  float lo[5], hi[5];
} sde_mlp_config;

sde_status sde_mlp_create(const sde_mlp_config *cfg, sde_mlp **out);
void sde_mlp_destroy(sde_mlp *mlp);
/* parameters per member */
int64_t sde_mlp_num_params(const sde_mlp *mlp);
/* copy one member's FP32 parameters in / out (device arrays of num_params) */
sde_status sde_mlp_set_params(sde_mlp *mlp, int32_t member, const float *params_dev, void *stream);
sde_status sde_mlp_get_params(sde_mlp *mlp, int32_t member, float *params_dev, void *stream);
/* features [n][5] from Eq. 1 parameter points (device array of sde_jj_point) */
sde_status sde_mlp_features(sde_mlp *mlp, const sde_jj_point *points_dev, int64_t n, float *X_dev,
                            void *stream);
/* forward pass of every member: mean_dev[b] = ensemble mean, spread_dev[b]
   = ensemble standard deviation (NULL allowed); X_dev [B][n_in] FP32.
   Networks of width 256 with 2..8 hidden layers and n_in <= 8 run one fused
   tensor-core kernel (the square hidden layers as tcgen05 MMAs of 128 points
   x 256 x 256 with BF16 operands and FP32 accumulators in tensor memory, the
   bias, SiLU and output layer in their epilogues); other shapes, or after
   sde_mlp_use_tensor_cores(mlp, 0), the CUDA-core kernels of the training
   path.  Asynchronous; an expired device wait of the tensor-core kernel is
   reported by sde_mlp_check. */
sde_status sde_mlp_forward(sde_mlp *mlp, const float *X_dev, int64_t B, float *mean_dev,
                           float *spread_dev, void *stream);
/* gradient of the mean-squared error of one member: grad_dev[num_params],
   loss_dev[1] (both device, FP32) */
sde_status sde_mlp_grad(sde_mlp *mlp, int32_t member, const float *X_dev, const float *y_dev,
                        int64_t B, float *grad_dev, float *loss_dev, void *stream);
/* select the tensor-core forward (enable != 0, the default where the shape
   allows it) or the CUDA-core one; SDE_ERR_UNSUPPORTED if the shape has no
   tensor-core path */
sde_status sde_mlp_use_tensor_cores(sde_mlp *mlp, int32_t enable);
/* synchronise the device and return SDE_ERR_TIMEOUT if a tensor-core forward
   kernel found a bounded wait expired since the last check (the status is
   then cleared; the affected outputs were not written) */
sde_status sde_mlp_check(sde_mlp *mlp);
/* change the Adam step size (learning-rate schedules); lr > 0 */
sde_status sde_mlp_set_lr(sde_mlp *mlp, float lr);
/* one Adam step of every member on the same batch; loss_dev[n_members] or NULL */
sde_status sde_mlp_train_step(sde_mlp *mlp, const float *X_dev, const float *y_dev, int64_t B,
                              float *loss_dev, void *stream);
/* one Adam step of every member on its own batch (bootstrap ensembles):
   X_dev [n_members][B][n_in], y_dev [n_members][B] */
sde_status sde_mlp_train_step_members(sde_mlp *mlp, const float *X_dev, const float *y_dev, int64_t B,
                                      float *loss_dev, void *stream);

/*
 * FP32 fused-multiply-add throughput probe (measurement infrastructure; the
 * paper has no counterpart).  Launches `grid` blocks of `block` threads
 * (block a multiple of 32, at most 256), each thread running eight
 * independent chains a <- 0.999 a + 0.001 for 16 * iters rounds: scalar FFMA
 * (packed = 0) or Blackwell's two-wide FFMA2 (packed = 1, two FMAs per
 * lane-instruction).  *flop_host (nullable) receives the FLOP the launch
 * executes (2 per FMA); the caller times the launch on `stream` with events
 * to obtain the FP32 peak that the integration kernels' rooflines use.
 * sink_dev: caller-owned device array of grid * block floats (written).
 * Errors: SDE_ERR_INVALID_ARG before any CUDA call; SDE_ERR_CUDA.
 */
sde_status sde_fp32_fma_probe(int32_t packed, int64_t iters, int32_t grid, int32_t block, float *sink_dev,
                              double *flop_host, void *stream);

/* Version of this ABI (major * 100 + minor).  102: the general-coupling GEMM
   forms (SDE_FLAG_GEMM_SINGLE_CTA, SDE_FLAG_GEMM_STREAM_K) and their
   sde_get_tuning values. */
int32_t sde_abi_version(void);

#ifdef __cplusplus
} /* extern "C" */
#endif

#endif /* SDE_GB300_H_ */
