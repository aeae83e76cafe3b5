// abi.cu -- the C ABI of include/sde.h: context creation, validation,
// autotuning, graph capture and the observables round trip.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <memory>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "kuramoto.h"

namespace sde {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

sde_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorName(e) + " (" +
            cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? SDE_ERR_NO_MEMORY : SDE_ERR_CUDA;
}

}  // namespace sde

using namespace sde;

struct sde_ctx {
  sde_config cfg{};
  int device = 0;
  int sm_count = 0;
  // ---- Josephson ----
  int n_points = 0;
  int P = 0;
  int64_t total_paths = 0;
  std::vector<int64_t> paths, steps, offsets;
  JJConsts *consts = nullptr;
  float *drive = nullptr;
  int64_t *offsets_dev = nullptr, *paths_dev = nullptr;  // per point (histograms)
  JJUnitList units[5];  // indexed by paths per thread (1, 2, 4)
  Moments *partials = nullptr;
  uint32_t *queue = nullptr;
  int block = 0, ilp = 0;
  // ---- Kuramoto ----
  KuramotoCtx *kur = nullptr;
  // ---- common ----
  sde_obs_row *obs = nullptr;
  int64_t n_obs_rows = 0;
  int64_t max_obs_rows = 0;
  uint32_t *err = nullptr;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  // graph cache
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  sde_run_desc gdesc{};
  bool gvalid = false;
};

namespace sde {

// Allocation-failure injection (sde_debug_fail_allocation): the number of
// allocations still to succeed before one fails, -1 = off.
static std::atomic<int> g_fail_countdown{-1};

bool injected_alloc_failure() {
  int n = g_fail_countdown.load();
  while (n >= 0) {
    if (g_fail_countdown.compare_exchange_weak(n, n - 1)) return n == 0;
  }
  return false;
}

void alloc_injection_disarm() { g_fail_countdown.store(-1); }

cudaError_t device_alloc(void **p, size_t bytes) {
  *p = nullptr;
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

}  // namespace sde

namespace {

template <class T>
cudaError_t dmalloc(T **p, size_t count) {
  if (count == 0) count = 1;
  return device_alloc((void **)p, sizeof(T) * count);
}

void free_ctx(sde_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  cudaFree(c->consts);
  cudaFree(c->drive);
  cudaFree(c->offsets_dev);
  cudaFree(c->paths_dev);
  for (auto &u : c->units) {
    cudaFree(u.units);
    cudaFree(u.point_range);
  }
  cudaFree(c->partials);
  cudaFree(c->queue);
  cudaFree(c->obs);
  cudaFree(c->err);
  kuramoto_destroy(c->kur);
  delete c;
}

// Work list: units of 32 * ilp paths, ordered by decreasing step count
// (longest-processing-time-first), ties by point index, so that the units of
// one point stay contiguous.
sde_status build_units(sde_ctx *c, int ilp) {
  JJUnitList &L = c->units[ilp];
  L.ilp = ilp;
  const int per = 32 * ilp;
  std::vector<int> order(c->n_points);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return c->steps[a] > c->steps[b]; });
  std::vector<JJUnit> units;
  L.point_range_h.assign(c->n_points, make_int2(0, 0));
  for (int p : order) {
    const int first = (int)units.size();
    for (int64_t b = 0; b < c->paths[p]; b += per) {
      JJUnit u;
      u.point = p;
      u.path_begin = (int32_t)b;
      u.n_paths = (int32_t)std::min<int64_t>(per, c->paths[p] - b);
      u.pad = 0;
      units.push_back(u);
    }
    L.point_range_h[p] = make_int2(first, (int)units.size());
  }
  L.n_units = (int32_t)units.size();
  SDE_CUDA_TRY(dmalloc(&L.units, units.size()));
  SDE_CUDA_TRY(dmalloc(&L.point_range, c->n_points));
  if (!units.empty())
    SDE_CUDA_TRY(cudaMemcpy(L.units, units.data(), sizeof(JJUnit) * units.size(),
                            cudaMemcpyHostToDevice));
  SDE_CUDA_TRY(cudaMemcpy(L.point_range, L.point_range_h.data(), sizeof(int2) * c->n_points,
                          cudaMemcpyHostToDevice));
  return SDE_OK;
}

// Launch variants: 1, 2, 4 = paths per thread; 11, 12, 14 = the same with
// fewer registers (64, 64, 96).  The work list depends on the paths per
// thread only.
int paths_per_thread(int variant) { return variant % 10; }

JJLaunchArgs jj_args(const sde_ctx *c, const sde_run_desc *r, int ilp) {
  JJLaunchArgs a{};
  a.consts = c->consts;
  a.units = c->units[paths_per_thread(ilp)].units;
  a.drive = c->drive;
  a.P = c->P;
  a.unit_begin = 0;
  a.unit_end = c->units[paths_per_thread(ilp)].n_units;
  a.queue = nullptr;
  a.partials = c->partials;
  a.err = c->err;
  a.st = JJState{r->x_in_dev, r->v_in_dev, r->w_in_dev, r->vsum_in_dev,
                 r->x_out_dev, r->v_out_dev, r->w_out_dev, r->vsum_out_dev};
  a.n_begin = r->n_begin;
  a.n_end = r->n_end;
  a.seed = c->cfg.seed;
  a.keys = philox_round_keys(c->cfg.seed);
  return a;
}

int persistent_grid(const sde_ctx *c, int ilp, int block) {
  const int per_sm = jj_max_blocks_per_sm(ilp, block, c->P);
  const int warps = block / 32;
  const int need = (c->units[paths_per_thread(ilp)].n_units + warps - 1) / warps;
  int grid = std::max(1, per_sm) * c->sm_count;
  return std::max(1, std::min(grid, need));
}

// Enqueue the work of one Josephson run (no graph).
// Events recorded while a stream is being captured must be external records
// to become event nodes of the graph.
cudaError_t record(cudaEvent_t e, cudaStream_t s, bool capturing) {
  return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

sde_status jj_enqueue(sde_ctx *c, const sde_run_desc *r, cudaStream_t s, int ilp, int block,
                      bool time_it, bool capturing = false) {
  JJLaunchArgs a = jj_args(c, r, ilp);
  const JJUnitList &L = c->units[paths_per_thread(ilp)];
  if (time_it) SDE_CUDA_TRY(record(c->ev0, s, capturing));
  if (c->cfg.schedule == SDE_SCHED_PERSISTENT) {
    if (L.n_units > 0) {
      SDE_CUDA_TRY(cudaMemsetAsync(c->queue, 0, sizeof(uint32_t), s));
      a.queue = c->queue;
      SDE_CUDA_TRY(jj_launch(a, ilp, block, persistent_grid(c, ilp, block), s));
    }
  } else {
    const int warps = block / 32;
    for (int p = 0; p < c->n_points; ++p) {
      const int2 pr = L.point_range_h[p];
      if (pr.y <= pr.x) continue;
      a.unit_begin = pr.x;
      a.unit_end = pr.y;
      const int grid = (pr.y - pr.x + warps - 1) / warps;
      SDE_CUDA_TRY(jj_launch(a, ilp, block, grid, s));
    }
  }
  if (time_it) SDE_CUDA_TRY(record(c->ev1, s, capturing));
  SDE_CUDA_TRY(jj_finalize(c->consts, L.point_range, c->n_points, c->partials, r->n_end, c->obs, s));
  return SDE_OK;
}

// Time each candidate launch shape on a short run (the first few hundred to
// 2048 steps) over the whole work list and keep the fastest.  Uses scratch state, so the caller's
// buffers are untouched.
sde_status jj_autotune(sde_ctx *c) {
  std::vector<std::pair<int, int>> cand;
  const bool fixed_block = c->cfg.block_threads > 0;
  const bool fixed_ilp = c->cfg.paths_per_thread > 0;
  const int blocks[] = {128, 256, 512};
  const int plain_blocks[] = {64, 128, 256, 512};
  std::vector<int> bl;
  if (fixed_block)
    bl.push_back(c->cfg.block_threads);
  else if (c->cfg.schedule == SDE_SCHED_PLAIN)
    bl.assign(std::begin(plain_blocks), std::end(plain_blocks));
  else
    bl.assign(std::begin(blocks), std::end(blocks));
  std::vector<int> il;
  if (fixed_ilp)
    il.push_back(c->cfg.paths_per_thread);
  else if (c->cfg.schedule == SDE_SCHED_PLAIN)
    il.push_back(1);  // the per-path kernel of Alg. 1: one thread per path
  else
    il = {2, 4, 12, 14};  // one path per thread never wins; it stays selectable
  // Euler-Maruyama kernels carry the variant code + 100
  const int scheme = (c->cfg.flags & SDE_FLAG_EULER) ? 100 : 0;
  for (int b : bl)
    for (int i : il) cand.push_back({b, i + scheme});
  if (cand.size() == 1) {
    c->block = cand[0].first;
    c->ilp = cand[0].second;
    return SDE_OK;
  }
  const int64_t np = std::max<int64_t>(std::min<int64_t>(c->total_paths, 1ll << 40), 1);
  float *x = nullptr, *v = nullptr;
  int32_t *w = nullptr;
  double *vs = nullptr;
  sde_status st = SDE_OK;
  cudaStream_t s = nullptr;
  auto fail = [&](cudaError_t e, const char *what) {
    st = cuda_fail(e, what);
  };
  cudaError_t e;
  if ((e = dmalloc(&x, np)) != cudaSuccess) fail(e, "autotune alloc");
  if (st == SDE_OK && (e = dmalloc(&v, np)) != cudaSuccess) fail(e, "autotune alloc");
  if (st == SDE_OK && (e = dmalloc(&w, np)) != cudaSuccess) fail(e, "autotune alloc");
  if (st == SDE_OK && (e = dmalloc(&vs, np)) != cudaSuccess) fail(e, "autotune alloc");
  if (st == SDE_OK && (e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess)
    fail(e, "autotune stream");
  if (st == SDE_OK) {
    cudaMemsetAsync(x, 0, sizeof(float) * np, s);
    cudaMemsetAsync(v, 0, sizeof(float) * np, s);
    sde_run_desc r{};
    r.n_begin = 0;
    int64_t max_steps = 0;
    for (auto S : c->steps) max_steps = std::max(max_steps, S);
    // every unit of the work list (the waves and the tail of the real run),
    // for 256 to 2048 steps: about 2^31 path-steps per trial at most
    const int64_t trial = std::min<int64_t>(2048, std::max<int64_t>(256, (1ll << 31) / np));
    r.n_end = std::min<int64_t>(max_steps, trial);
    r.x_in_dev = x;
    r.v_in_dev = v;
    r.x_out_dev = x;
    r.v_out_dev = v;
    r.w_out_dev = w;
    r.vsum_out_dev = vs;
    float best = 1e30f;
    for (auto &cd : cand) {
      float ms_min = 1e30f;
      for (int rep = 0; rep < 3 && st == SDE_OK; ++rep) {
        st = jj_enqueue(c, &r, s, cd.second, cd.first, true, false);
        if (st != SDE_OK) break;
        if ((e = cudaEventSynchronize(c->ev1)) != cudaSuccess) {
          fail(e, "autotune sync");
          break;
        }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        if (rep > 0) ms_min = std::min(ms_min, ms);
      }
      if (st != SDE_OK) break;
      if (ms_min < best) {
        best = ms_min;
        c->block = cd.first;
        c->ilp = cd.second;
      }
    }
    if (st == SDE_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) fail(e, "autotune sync");
    if (st == SDE_OK) cudaMemset(c->err, 0, sizeof(uint32_t));
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(x);
  cudaFree(v);
  cudaFree(w);
  cudaFree(vs);
  return st;
}

// Host-side checks of a Josephson configuration (no CUDA call).
sde_status validate_josephson(const sde_config *cfg) {
  SDE_CHECK_ARG(cfg->n_points >= 1, "n_points must be >= 1");
  SDE_CHECK_ARG(cfg->points && cfg->paths && cfg->steps, "points/paths/steps must be non-NULL");
  SDE_CHECK_ARG(cfg->steps_per_period >= 1 && cfg->steps_per_period <= 4096,
                "steps_per_period must be in [1, 4096]");
  SDE_CHECK_ARG(cfg->schedule == SDE_SCHED_PERSISTENT || cfg->schedule == SDE_SCHED_PLAIN,
                "unknown schedule");
  SDE_CHECK_ARG(cfg->block_threads == 0 ||
                    (cfg->block_threads >= 32 && cfg->block_threads <= 512 &&
                     cfg->block_threads % 32 == 0),
                "block_threads must be 0 or a multiple of 32 in [32, 512]");
  SDE_CHECK_ARG(cfg->paths_per_thread == 0 || cfg->paths_per_thread == 1 || cfg->paths_per_thread == 2 ||
                    cfg->paths_per_thread == 4 || cfg->paths_per_thread == 11 || cfg->paths_per_thread == 12 ||
                    cfg->paths_per_thread == 14,
                "paths_per_thread must be 0, 1, 2, 4, 11, 12 or 14");
  int64_t off = 0;
  for (int p = 0; p < cfg->n_points; ++p) {
    const sde_jj_point &q = cfg->points[p];
    SDE_CHECK_ARG(isfinite(q.gamma) && isfinite(q.a) && isfinite(q.omega) && isfinite(q.f) &&
                      isfinite(q.D),
                  "point parameters must be finite");
    SDE_CHECK_ARG(q.omega > 0.0, "omega must be > 0");
    SDE_CHECK_ARG(q.gamma > 0.0, "gamma must be > 0");
    SDE_CHECK_ARG(q.D >= 0.0, "D must be >= 0");
    SDE_CHECK_ARG(cfg->paths[p] >= 0 && cfg->paths[p] < (1ll << 31), "paths out of range");
    SDE_CHECK_ARG(cfg->steps[p] >= 0 && cfg->steps[p] <= (1ll << 33), "steps out of range");
    off += cfg->paths[p];
  }
  SDE_CHECK_ARG(off < (1ll << 40), "total paths too large");
  return SDE_OK;
}

sde_status create_josephson(sde_ctx *c, const sde_config *cfg) {
  const sde_status vs = validate_josephson(cfg);
  if (vs != SDE_OK) return vs;
  c->n_points = cfg->n_points;
  c->P = cfg->steps_per_period;
  c->paths.resize(c->n_points);
  c->steps.resize(c->n_points);
  c->offsets.resize(c->n_points);
  int64_t off = 0;
  for (int p = 0; p < c->n_points; ++p) {
    c->paths[p] = cfg->paths[p];
    c->steps[p] = cfg->steps[p];
    c->offsets[p] = off;
    off += cfg->paths[p];
  }
  c->total_paths = off;
  SDE_CUDA_TRY(jj_configure());

  // the point and step tables are needed only by the prepare kernel: freed
  // on every way out of this block
  struct DevFree {
    void operator()(void *p) const { cudaFree(p); }
  };
  sde_jj_point *pts_raw = nullptr;
  int64_t *steps_raw = nullptr;
  SDE_CUDA_TRY(dmalloc(&pts_raw, c->n_points));
  std::unique_ptr<sde_jj_point, DevFree> pts(pts_raw);
  SDE_CUDA_TRY(dmalloc(&steps_raw, c->n_points));
  std::unique_ptr<int64_t, DevFree> steps(steps_raw);
  SDE_CUDA_TRY(dmalloc(&c->offsets_dev, c->n_points));
  SDE_CUDA_TRY(dmalloc(&c->paths_dev, c->n_points));
  SDE_CUDA_TRY(dmalloc(&c->consts, c->n_points));
  SDE_CUDA_TRY(dmalloc(&c->drive, c->P));
  SDE_CUDA_TRY(cudaMemcpy(pts.get(), cfg->points, sizeof(sde_jj_point) * c->n_points, cudaMemcpyHostToDevice));
  SDE_CUDA_TRY(cudaMemcpy(steps.get(), c->steps.data(), 8 * c->n_points, cudaMemcpyHostToDevice));
  SDE_CUDA_TRY(cudaMemcpy(c->offsets_dev, c->offsets.data(), 8 * c->n_points, cudaMemcpyHostToDevice));
  SDE_CUDA_TRY(cudaMemcpy(c->paths_dev, c->paths.data(), 8 * c->n_points, cudaMemcpyHostToDevice));
  SDE_CUDA_TRY(jj_prepare(pts.get(), c->n_points, c->P, steps.get(), c->offsets_dev, c->paths_dev, c->consts,
                          c->drive, 0));
  SDE_CUDA_TRY(cudaDeviceSynchronize());

  int32_t max_units = 0;
  for (int ilp : {1, 2, 4}) {
    sde_status st = build_units(c, ilp);
    if (st != SDE_OK) return st;
    max_units = std::max(max_units, c->units[ilp].n_units);
  }
  SDE_CUDA_TRY(dmalloc(&c->partials, max_units));
  SDE_CUDA_TRY(dmalloc(&c->queue, 1));
  c->max_obs_rows = c->n_points;
  SDE_CUDA_TRY(dmalloc(&c->obs, c->max_obs_rows));
  SDE_CUDA_TRY(cudaMemset(c->obs, 0, sizeof(sde_obs_row) * c->max_obs_rows));
  return jj_autotune(c);
}

sde_status run_graph(sde_ctx *c, const sde_run_desc *r, cudaStream_t s) {
  const bool same = c->gvalid && memcmp(&c->gdesc, r, sizeof(sde_run_desc)) == 0;
  if (!same) {
    if (c->gexec) {
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
    c->gvalid = false;
    cudaGraph_t g = nullptr;
    SDE_CUDA_TRY(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    sde_status st = jj_enqueue(c, r, c->cap_stream, c->ilp, c->block, true, true);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != SDE_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c->gdesc = *r;
    c->gvalid = true;
  }
  SDE_CUDA_TRY(cudaGraphLaunch(c->gexec, s));
  return SDE_OK;
}

}  // namespace

extern "C" {

int32_t sde_abi_version(void) { return 102; }

const char *sde_last_error(void) { return g_last_error.c_str(); }

sde_status sde_create(const sde_config *cfg, sde_ctx **out) {
  clear_error();
  if (!out) {
    set_error("invalid argument: out is NULL");
    return SDE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  SDE_CHECK_ARG(cfg != nullptr, "cfg is NULL");
  // the configuration is checked on the host before any CUDA call
  sde_status vs = SDE_OK;
  switch (cfg->model) {
    case SDE_JOSEPHSON:
      vs = validate_josephson(cfg);
      break;
    case SDE_KURAMOTO_MEANFIELD:
    case SDE_KURAMOTO_PAIRWISE:
    case SDE_KURAMOTO_GENERAL:
    case SDE_KURAMOTO_GENERAL_FP32:
      vs = kuramoto_validate(cfg);
      break;
    default:
      set_error("invalid argument: unknown model");
      vs = SDE_ERR_INVALID_ARG;
  }
  if (vs != SDE_OK) return vs;
  sde_ctx *c = injected_alloc_failure() ? nullptr : new (std::nothrow) sde_ctx();
  if (!c) {
    alloc_injection_disarm();
    set_error("host allocation failed");
    return SDE_ERR_NO_MEMORY;
  }
  c->cfg = *cfg;
  c->cfg.points = nullptr;
  c->cfg.paths = nullptr;
  c->cfg.steps = nullptr;
  sde_status st = SDE_OK;
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess) st = cuda_fail(e, "cudaGetDevice");
  if (st == SDE_OK &&
      (e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess)
    st = cuda_fail(e, "cudaDeviceGetAttribute");
  if (st == SDE_OK && (e = dmalloc(&c->err, 1)) != cudaSuccess) st = cuda_fail(e, "cudaMalloc");
  if (st == SDE_OK && (e = cudaMemset(c->err, 0, sizeof(uint32_t))) != cudaSuccess)
    st = cuda_fail(e, "cudaMemset");
  if (st == SDE_OK && (e = cudaEventCreate(&c->ev0)) != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");
  if (st == SDE_OK && (e = cudaEventCreate(&c->ev1)) != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");
  if (st == SDE_OK && (e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    st = cuda_fail(e, "cudaStreamCreate");
  if (st == SDE_OK) {
    switch (cfg->model) {
      case SDE_JOSEPHSON:
        st = create_josephson(c, cfg);
        break;
      case SDE_KURAMOTO_MEANFIELD:
      case SDE_KURAMOTO_PAIRWISE:
      case SDE_KURAMOTO_GENERAL:
      case SDE_KURAMOTO_GENERAL_FP32:
        st = kuramoto_create(cfg, c->sm_count, c->err, &c->kur);
        break;
      default:
        set_error("invalid argument: unknown model");
        st = SDE_ERR_INVALID_ARG;
    }
  }
  alloc_injection_disarm();
  if (st != SDE_OK) {
    std::string msg = g_last_error;
    free_ctx(c);
    set_error(msg);
    return st;
  }
  *out = c;
  return SDE_OK;
}

sde_status sde_run_ensemble(sde_ctx *c, const sde_run_desc *r, void *stream) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr && r != nullptr, "ctx and run must be non-NULL");
  SDE_CHECK_ARG(r->n_begin >= 0 && r->n_end >= r->n_begin, "need 0 <= n_begin <= n_end");
  SDE_CHECK_ARG(r->n_end <= (1ll << 33), "n_end out of range");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = -1;
  SDE_CUDA_TRY(cudaGetDevice(&dev));
  SDE_CHECK_ARG(dev == c->device, "current device differs from the context's device");
  if (c->cfg.model == SDE_JOSEPHSON) {
    if (c->total_paths > 0) {
      SDE_CHECK_ARG(r->x_in_dev && r->v_in_dev && r->x_out_dev && r->v_out_dev && r->w_out_dev &&
                        r->vsum_out_dev,
                    "Josephson run needs x_in, v_in, x_out, v_out, w_out and vsum_out");
    }
    sde_status st;
    if (c->cfg.flags & SDE_FLAG_NO_GRAPH)
      st = jj_enqueue(c, r, s, c->ilp, c->block, true);
    else
      st = run_graph(c, r, s);
    if (st != SDE_OK) return st;
    c->n_obs_rows = c->n_points;
  } else {
    int64_t rows = 0;
    sde_status st = kuramoto_run(c->kur, r, s, c->ev0, c->ev1, c->obs, &c->obs, &c->max_obs_rows, &rows);
    if (st != SDE_OK) return st;
    c->n_obs_rows = rows;
  }
  c->last_stream = s;
  c->timed = true;
  return SDE_OK;
}

sde_status sde_observables(sde_ctx *c, sde_obs_row *rows, int64_t capacity, int64_t *n_rows) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  SDE_CHECK_ARG(capacity >= 0 && (rows != nullptr || capacity == 0), "rows/capacity");
  SDE_CUDA_TRY(cudaStreamSynchronize(c->last_stream));
  const int64_t n = std::min<int64_t>(capacity, c->n_obs_rows);
  if (n > 0) SDE_CUDA_TRY(cudaMemcpy(rows, c->obs, sizeof(sde_obs_row) * n, cudaMemcpyDeviceToHost));
  if (n_rows) *n_rows = c->n_obs_rows;
  uint32_t err = 0;
  SDE_CUDA_TRY(cudaMemcpy(&err, c->err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  // a latched device status is reported once, then cleared for later runs
  if (err) SDE_CUDA_TRY(cudaMemset(c->err, 0, sizeof(uint32_t)));
  if (err & kErrTimeout) {
    set_error("a bounded device wait expired");
    return SDE_ERR_TIMEOUT;
  }
  if (err & kErrNonFinite) {
    set_error("a kernel produced a non-finite state");
    return SDE_ERR_NUMERIC;
  }
  return SDE_OK;
}

void sde_destroy(sde_ctx *c) { free_ctx(c); }

sde_status sde_set_wait_limit(sde_ctx *c, uint64_t ns) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  // Josephson kernels have no device waits: nothing to set there
  if (c->kur) kuramoto_set_wait_limit(c->kur, ns == 0 ? 1000000000ull : ns);
  return SDE_OK;
}

void sde_debug_fail_allocation(int32_t nth) { g_fail_countdown.store(nth >= 1 ? nth - 1 : -1); }

sde_status sde_get_tuning(const sde_ctx *c, int32_t *block, int32_t *ilp, int32_t *cluster) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  if (c->kur) {
    kuramoto_tuning(c->kur, block, ilp, cluster);
    return SDE_OK;
  }
  if (block) *block = c->block;
  if (ilp) *ilp = c->ilp % 100;
  if (cluster) *cluster = 1;
  return SDE_OK;
}

sde_status sde_last_kernel_stats(sde_ctx *c, float *mean_ms, float *total_ms, int64_t *launches) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  SDE_CHECK_ARG(c->timed, "no run has been timed yet");
  if (c->kur && kuramoto_kernel_stats(c->kur, mean_ms, total_ms, launches)) return SDE_OK;
  float ms = 0.0f;
  SDE_CUDA_TRY(cudaEventSynchronize(c->ev1));
  SDE_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  if (mean_ms) *mean_ms = ms;
  if (total_ms) *total_ms = ms;
  if (launches) *launches = 1;
  return SDE_OK;
}

sde_status sde_last_kernel_ms(sde_ctx *c, float *ms) {
  clear_error();
  SDE_CHECK_ARG(ms != nullptr, "ms is NULL");
  return sde_last_kernel_stats(c, ms, nullptr, nullptr);
}

sde_status sde_position_histogram(sde_ctx *c, const int32_t *w_dev, int32_t w_lo, int32_t nbins,
                                  unsigned long long *counts_dev, void *stream) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr && c->cfg.model == SDE_JOSEPHSON, "needs a Josephson context");
  SDE_CHECK_ARG(nbins >= 1 && nbins <= 8192, "nbins must be in [1, 8192]");
  SDE_CHECK_ARG(counts_dev != nullptr, "counts is NULL");
  SDE_CHECK_ARG(w_dev != nullptr || c->total_paths == 0, "w is NULL");
  int64_t max_paths = 0;
  for (auto p : c->paths) max_paths = std::max(max_paths, p);
  SDE_CUDA_TRY(winding_hist(w_dev, c->offsets_dev, c->paths_dev, c->n_points, max_paths, w_lo, nbins,
                            counts_dev, c->sm_count, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_phase_histogram(const float *phi_dev, int64_t n, int32_t nbins, unsigned long long *counts_dev,
                               void *stream) {
  clear_error();
  SDE_CHECK_ARG(n >= 0 && nbins >= 1 && nbins <= 8192, "need n >= 0 and nbins in [1, 8192]");
  SDE_CHECK_ARG(counts_dev != nullptr && (phi_dev != nullptr || n == 0), "phi and counts must be non-NULL");
  int dev = 0, sms = 0;
  SDE_CUDA_TRY(cudaGetDevice(&dev));
  SDE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SDE_CUDA_TRY(phase_hist(phi_dev, n, nbins, counts_dev, sms, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_set_coupling(sde_ctx *c, const float *K_dev, void *stream) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  SDE_CHECK_ARG(c->kur != nullptr, "sde_set_coupling applies to Kuramoto contexts");
  return kuramoto_set_coupling(c->kur, K_dev, (cudaStream_t)stream);
}

sde_status sde_kuramoto_coupling(sde_ctx *c, const float *phi_dev, float *out_dev, void *stream) {
  clear_error();
  SDE_CHECK_ARG(c != nullptr, "ctx is NULL");
  SDE_CHECK_ARG(c->kur != nullptr, "sde_kuramoto_coupling applies to Kuramoto contexts");
  return kuramoto_coupling(c->kur, phi_dev, out_dev, (cudaStream_t)stream);
}

sde_status sde_philox4x32_10(const uint32_t *ctr, uint64_t seed, uint32_t *out, int64_t n,
                             void *stream) {
  clear_error();
  SDE_CHECK_ARG(n >= 0, "n must be >= 0");
  SDE_CHECK_ARG(n == 0 || (ctr && out), "ctr and out must be non-NULL");
  SDE_CHECK_ARG(((uintptr_t)ctr % 16) == 0 && ((uintptr_t)out % 16) == 0,
                "ctr and out must be 16-byte aligned");
  SDE_CUDA_TRY(philox_fill(ctr, seed, out, n, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_box_muller(const uint32_t *ctr, uint64_t seed, float *z, int64_t n, void *stream) {
  clear_error();
  SDE_CHECK_ARG(n >= 0, "n must be >= 0");
  SDE_CHECK_ARG(n == 0 || (ctr && z), "ctr and z must be non-NULL");
  SDE_CHECK_ARG(((uintptr_t)ctr % 16) == 0 && ((uintptr_t)z % 16) == 0,
                "ctr and z must be 16-byte aligned");
  SDE_CUDA_TRY(box_muller_fill(ctr, seed, z, n, (cudaStream_t)stream));
  return SDE_OK;
}

sde_status sde_box_muller_words(const uint32_t *w, int64_t n_pairs, int32_t variant, float *z, void *stream) {
  clear_error();
  SDE_CHECK_ARG(n_pairs >= 0, "n_pairs must be >= 0");
  SDE_CHECK_ARG(variant == 0 || variant == 1, "variant must be 0 or 1");
  SDE_CHECK_ARG(n_pairs == 0 || (w && z), "w and z must be non-NULL");
  SDE_CHECK_ARG(((uintptr_t)w % 8) == 0 && ((uintptr_t)z % 8) == 0, "w and z must be 8-byte aligned");
  SDE_CUDA_TRY(box_muller_words(w, n_pairs, variant, z, (cudaStream_t)stream));
  return SDE_OK;
}

}  // extern "C"
