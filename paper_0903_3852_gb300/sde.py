"""Thin ctypes binding of the C ABI in include/sde.h (libsde_gb300.so).

Argument marshalling only: every step of the integration runs in the CUDA
library.  Device buffers are torch tensors on the current CUDA device; their
data pointers and the current torch stream are passed through unchanged.  There
is no CPU fallback: if the library is missing this module raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsde_gb300.so")

SDE_OK = 0
SDE_ERR_INVALID_ARG, SDE_ERR_CUDA, SDE_ERR_NO_MEMORY, SDE_ERR_TIMEOUT, SDE_ERR_UNSUPPORTED, SDE_ERR_NUMERIC = 1, 2, 3, 4, 5, 6
STATUS_NAMES = {0: "SDE_OK", 1: "SDE_ERR_INVALID_ARG", 2: "SDE_ERR_CUDA", 3: "SDE_ERR_NO_MEMORY",
                4: "SDE_ERR_TIMEOUT", 5: "SDE_ERR_UNSUPPORTED", 6: "SDE_ERR_NUMERIC"}

SDE_JOSEPHSON = 0
SDE_KURAMOTO_MEANFIELD = 1
SDE_KURAMOTO_PAIRWISE = 2
SDE_KURAMOTO_GENERAL = 3
SDE_KURAMOTO_GENERAL_FP32 = 4

SDE_SCHED_PERSISTENT = 0
SDE_SCHED_PLAIN = 1
SDE_SCHED_GRID = 2

SDE_FLAG_NO_GRAPH = 1
SDE_FLAG_TIME_KERNELS = 2
SDE_FLAG_FUSED = 4
SDE_FLAG_EULER = 8
SDE_FLAG_ASYNC_EXCHANGE = 16
SDE_FLAG_GEMM_SINGLE_CTA = 32
SDE_FLAG_GEMM_STREAM_K = 64


class SDEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class JJPoint(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("a", ctypes.c_double), ("omega", ctypes.c_double),
                ("f", ctypes.c_double), ("D", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("schedule", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("n_points", ctypes.c_int32), ("steps_per_period", ctypes.c_int32),
                ("points", ctypes.POINTER(JJPoint)), ("paths", ctypes.POINTER(ctypes.c_int64)),
                ("steps", ctypes.POINTER(ctypes.c_int64)),
                ("n_osc", ctypes.c_int64), ("n_replicas", ctypes.c_int64), ("K", ctypes.c_double),
                ("D", ctypes.c_double), ("dt", ctypes.c_double), ("sample_every", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("paths_per_thread", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("cluster_ctas", ctypes.c_int32)]


class RunDesc(ctypes.Structure):
    _fields_ = [("n_begin", ctypes.c_int64), ("n_end", ctypes.c_int64),
                ("x_in_dev", ctypes.c_void_p), ("v_in_dev", ctypes.c_void_p),
                ("w_in_dev", ctypes.c_void_p), ("vsum_in_dev", ctypes.c_void_p),
                ("x_out_dev", ctypes.c_void_p), ("v_out_dev", ctypes.c_void_p),
                ("w_out_dev", ctypes.c_void_p), ("vsum_out_dev", ctypes.c_void_p),
                ("phi_in_dev", ctypes.c_void_p), ("phi_out_dev", ctypes.c_void_p),
                ("omega_dev", ctypes.c_void_p), ("r_out_dev", ctypes.c_void_p)]


class ObsRow(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double), ("var", ctypes.c_double), ("se", ctypes.c_double),
                ("count", ctypes.c_double), ("t", ctypes.c_double)]


class MlpConfig(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int32), ("hidden", ctypes.c_int32), ("n_hidden", ctypes.c_int32),
                ("n_members", ctypes.c_int32), ("max_batch", ctypes.c_int64), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("lo", ctypes.c_float * 5), ("hi", ctypes.c_float * 5)]


_lib = None

# (name, restype, argtypes) of every exported symbol declared in include/sde.h
_VP = ctypes.c_void_p
SIGNATURES = [
    ("sde_create", ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_VP)]),
    ("sde_run_ensemble", ctypes.c_int, [_VP, ctypes.POINTER(RunDesc), _VP]),
    ("sde_observables", ctypes.c_int, [_VP, ctypes.POINTER(ObsRow), ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("sde_destroy", None, [_VP]),
    ("sde_last_error", ctypes.c_char_p, []),
    ("sde_get_tuning", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    ("sde_last_kernel_ms", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    ("sde_last_kernel_stats", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int64)]),
    ("sde_philox4x32_10", ctypes.c_int, [_VP, ctypes.c_uint64, _VP, ctypes.c_int64, _VP]),
    ("sde_box_muller", ctypes.c_int, [_VP, ctypes.c_uint64, _VP, ctypes.c_int64, _VP]),
    ("sde_abi_version", ctypes.c_int32, []),
    ("sde_set_coupling", ctypes.c_int, [_VP, _VP, _VP]),
    ("sde_position_histogram", ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.c_int32, _VP, _VP]),
    ("sde_phase_histogram", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP]),
    ("sde_mlp_create", ctypes.c_int, [ctypes.POINTER(MlpConfig), ctypes.POINTER(_VP)]),
    ("sde_mlp_destroy", None, [_VP]),
    ("sde_mlp_num_params", ctypes.c_int64, [_VP]),
    ("sde_mlp_set_params", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP]),
    ("sde_mlp_get_params", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP]),
    ("sde_mlp_features", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("sde_mlp_forward", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    ("sde_mlp_grad", ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, ctypes.c_int64, _VP, _VP, _VP]),
    ("sde_mlp_train_step", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("sde_mlp_set_lr", ctypes.c_int, [_VP, ctypes.c_float]),
    ("sde_mlp_train_step_members", ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, _VP, _VP]),
    ("sde_kuramoto_coupling", ctypes.c_int, [_VP, _VP, _VP, _VP]),
    ("sde_josephson_run_noalloc", ctypes.c_int,
     [ctypes.POINTER(JJPoint), ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
      ctypes.c_int64, ctypes.c_int64] + [_VP] * 9 + [_VP]),
    ("sde_box_muller_words", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int32, _VP, _VP]),
    ("sde_set_wait_limit", ctypes.c_int, [_VP, ctypes.c_uint64]),
    ("sde_mlp_use_tensor_cores", ctypes.c_int, [_VP, ctypes.c_int32]),
    ("sde_mlp_check", ctypes.c_int, [_VP]),
    ("sde_debug_fail_allocation", None, [ctypes.c_int32]),
    ("sde_fp32_fma_probe", ctypes.c_int,
     [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_double), _VP]),
    ("sde_josephson_run_fp64", ctypes.c_int,
     [ctypes.POINTER(JJPoint), ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
      ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64] + [_VP] * 7 + [_VP]),
]

NOALLOC_MAX_PATHS = 1 << 20


def lib():
    """Load libsde_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsde_gb300.so is not built (%s); run "
                               "python -m paper_0903_3852_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != SDE_OK:
        raise SDEError(status, lib().sde_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    import torch
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "need contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def philox4x32_10(ctr, seed, stream=None):
    """ctr: (n, 4) int32/uint32 CUDA tensor -> (n, 4) int32 tensor of Philox words (bit patterns)."""
    import torch
    assert ctr.dim() == 2 and ctr.shape[1] == 4
    out = torch.empty_like(ctr)
    _check(lib().sde_philox4x32_10(_ptr(ctr), seed, _ptr(out), ctr.shape[0], _stream(stream)))
    return out


def box_muller(ctr, seed, stream=None):
    """ctr: (n, 4) int32 CUDA tensor -> (n, 4) float32 Gaussians as the integrators draw them."""
    import torch
    assert ctr.dim() == 2 and ctr.shape[1] == 4
    z = torch.empty(ctr.shape, dtype=torch.float32, device=ctr.device)
    _check(lib().sde_box_muller(_ptr(ctr), seed, _ptr(z), ctr.shape[0], _stream(stream)))
    return z


class Ensemble:
    """An sde_ctx: one configured ensemble (Josephson points or Kuramoto replicas)."""

    def __init__(self, cfg: Config, keep=()):
        self._keep = keep
        h = _VP()
        _check(lib().sde_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.cfg = cfg

    @classmethod
    def josephson(cls, points, paths, steps, seed, steps_per_period=200,
                  schedule=SDE_SCHED_PERSISTENT, block_threads=0, paths_per_thread=0, flags=0):
        n = len(points)
        pts = (JJPoint * n)(*[JJPoint(p["gamma"], p["a"], p["omega"], p["f"], p["D"]) for p in points])
        pa = np.ascontiguousarray(np.asarray(paths, dtype=np.int64))
        st = np.ascontiguousarray(np.asarray(steps, dtype=np.int64))
        cfg = Config()
        cfg.model = SDE_JOSEPHSON
        cfg.schedule = schedule
        cfg.seed = seed
        cfg.n_points = n
        cfg.steps_per_period = steps_per_period
        cfg.points = ctypes.cast(pts, ctypes.POINTER(JJPoint))
        cfg.paths = pa.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        cfg.steps = st.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        cfg.block_threads = block_threads
        cfg.paths_per_thread = paths_per_thread
        cfg.flags = flags
        e = cls(cfg, keep=(pts, pa, st))
        e.n_points = n
        e.paths = pa.copy()
        e.steps = st.copy()
        e.total_paths = int(pa.sum())
        return e

    @classmethod
    def kuramoto(cls, model, n_osc, n_replicas, K, D, dt, seed, sample_every=100, block_threads=0,
                 flags=0, cluster_ctas=0, schedule=SDE_SCHED_PERSISTENT):
        cfg = Config()
        cfg.model = model
        cfg.schedule = schedule
        cfg.seed = seed
        cfg.n_osc = n_osc
        cfg.n_replicas = n_replicas
        cfg.K = K
        cfg.D = D
        cfg.dt = dt
        cfg.sample_every = sample_every
        cfg.block_threads = block_threads
        cfg.flags = flags
        cfg.cluster_ctas = cluster_ctas
        e = cls(cfg)
        e.n_osc, e.n_replicas, e.sample_every = n_osc, n_replicas, sample_every
        return e

    def run_josephson(self, n_begin, n_end, x_in, v_in, x_out, v_out, w_out, vsum_out, w_in=None,
                      vsum_in=None, stream=None):
        r = RunDesc()
        r.n_begin, r.n_end = n_begin, n_end
        r.x_in_dev, r.v_in_dev = _ptr(x_in), _ptr(v_in)
        r.w_in_dev, r.vsum_in_dev = _ptr(w_in), _ptr(vsum_in)
        r.x_out_dev, r.v_out_dev = _ptr(x_out), _ptr(v_out)
        r.w_out_dev, r.vsum_out_dev = _ptr(w_out), _ptr(vsum_out)
        _check(lib().sde_run_ensemble(self._h, ctypes.byref(r), _stream(stream)))

    def run_kuramoto(self, n_begin, n_end, phi_in, phi_out, omega, r_out=None, stream=None):
        r = RunDesc()
        r.n_begin, r.n_end = n_begin, n_end
        r.phi_in_dev, r.phi_out_dev, r.omega_dev = _ptr(phi_in), _ptr(phi_out), _ptr(omega)
        r.r_out_dev = _ptr(r_out)
        _check(lib().sde_run_ensemble(self._h, ctypes.byref(r), _stream(stream)))

    def position_histogram(self, w, w_lo, nbins, stream=None):
        """Per-point counts of the winding count w: (n_points, nbins + 2) int64
        tensor [below, w_lo .. w_lo + nbins - 1, above]."""
        import torch
        counts = torch.empty((self.n_points, nbins + 2), dtype=torch.int64, device="cuda")
        _check(lib().sde_position_histogram(self._h, _ptr(w), w_lo, nbins, _ptr(counts), _stream(stream)))
        return counts

    def set_coupling(self, K, stream=None):
        """K: (N, N) float32 CUDA tensor, row i = receiving oscillator."""
        _check(lib().sde_set_coupling(self._h, _ptr(K), _stream(stream)))

    def coupling(self, phi, stream=None):
        """Coupling sums sum_j K_ij sin(phi_j - phi_i) for phi of shape (R, N)."""
        import torch
        out = torch.empty_like(phi)
        _check(lib().sde_kuramoto_coupling(self._h, _ptr(phi), _ptr(out), _stream(stream)))
        return out

    def observables(self, capacity=None):
        """Synchronise and return the FP64 observables as a structured numpy array
        with fields mean, var, se, count, t."""
        n = ctypes.c_int64()
        _check(lib().sde_observables(self._h, None, 0, ctypes.byref(n)))
        cap = n.value if capacity is None else capacity
        rows = (ObsRow * max(cap, 1))()
        _check(lib().sde_observables(self._h, rows, cap, ctypes.byref(n)))
        dt = np.dtype([("mean", "f8"), ("var", "f8"), ("se", "f8"), ("count", "f8"), ("t", "f8")])
        out = np.frombuffer(bytearray(rows)[:ctypes.sizeof(ObsRow) * min(cap, n.value)], dtype=dt)
        return out.copy()

    def tuning(self):
        """(threads per block, paths or oscillators per thread, CTAs per replica)."""
        b, i, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().sde_get_tuning(self._h, ctypes.byref(b), ctypes.byref(i), ctypes.byref(c)))
        return b.value, i.value, c.value

    def last_kernel_ms(self):
        ms = ctypes.c_float()
        _check(lib().sde_last_kernel_ms(self._h, ctypes.byref(ms)))
        return ms.value

    def last_kernel_stats(self):
        """(mean ms per launch, total ms, launches) of the dominant kernel in the last run."""
        m, t, n = ctypes.c_float(), ctypes.c_float(), ctypes.c_int64()
        _check(lib().sde_last_kernel_stats(self._h, ctypes.byref(m), ctypes.byref(t), ctypes.byref(n)))
        return m.value, t.value, n.value

    def set_wait_limit(self, ns):
        """Limit (ns) of the bounded device waits of later launches; 0 = the
        default one second."""
        _check(lib().sde_set_wait_limit(self._h, ns))

    def close(self):
        if getattr(self, "_h", None):
            lib().sde_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_buffers(named):
    """Each (name, tensor, dtype, n) must be a contiguous tensor of that dtype
    with at least n elements on the current CUDA device; raises ValueError
    before anything reaches the GPU (sizes first, then types, then devices)."""
    import torch
    for name, t, dtype, n in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.numel() < n:
            raise ValueError("%s holds %d elements, fewer than the %d required" % (name, t.numel(), n))
    for name, t, dtype, n in named:
        if t.dtype != dtype:
            raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
    for name, t, dtype, n in named:
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise ValueError("%s must be on the current CUDA device, got %s" % (name, t.device))


def josephson_run_noalloc(point, steps_per_period, n_paths, total_steps, seed, n_begin, n_end,
                          x_in, v_in, x_out, v_out, w_out, vsum_out, obs_out, w_in=None, vsum_in=None,
                          stream=None):
    """sde_josephson_run_noalloc: one parameter point, no device allocation by the
    library (scratch lives in a fixed static array of NOALLOC_MAX_PATHS / 32
    partials).  obs_out: a CUDA tensor of 5 float64 (one sde_obs_row)."""
    import torch
    # The C entry point sees bare pointers and cannot check buffer sizes: a
    # short or mistyped buffer would be read or written past its end on the
    # GPU, so every buffer is checked here before the call.
    n = int(n_paths)
    if n < 0:
        raise ValueError("n_paths must be >= 0")
    need = [("x_in", x_in, torch.float32, n), ("v_in", v_in, torch.float32, n),
            ("x_out", x_out, torch.float32, n), ("v_out", v_out, torch.float32, n),
            ("w_out", w_out, torch.int32, n), ("vsum_out", vsum_out, torch.float64, n),
            ("obs_out", obs_out, torch.float64, 5)]
    if w_in is not None:
        need.append(("w_in", w_in, torch.int32, n))
    if vsum_in is not None:
        need.append(("vsum_in", vsum_in, torch.float64, n))
    _check_buffers(need)
    p = JJPoint(point["gamma"], point["a"], point["omega"], point["f"], point["D"])
    _check(lib().sde_josephson_run_noalloc(
        ctypes.byref(p), steps_per_period, n_paths, total_steps, seed, n_begin, n_end,
        _ptr(x_in), _ptr(v_in), _ptr(w_in), _ptr(vsum_in), _ptr(x_out), _ptr(v_out), _ptr(w_out),
        _ptr(vsum_out), _ptr(obs_out), _stream(stream)))


def box_muller_words(w, variant=0, stream=None):
    """sde_box_muller_words: Gaussians from given word pairs; w is a CUDA int32/uint32
    tensor of shape (n, 2); returns a float32 tensor (n, 2)."""
    import torch
    assert w.is_cuda and w.dim() == 2 and w.shape[1] == 2 and w.element_size() == 4
    w = w.contiguous()
    z = torch.empty(w.shape, dtype=torch.float32, device=w.device)
    _check(lib().sde_box_muller_words(_ptr(w), w.shape[0], variant, _ptr(z), _stream(stream)))
    return z


def josephson_run_fp64(point, steps_per_period, total_steps, seed, n_begin, n_end, x_in, v_in, x_out, v_out,
                       vsum_in=None, vsum_out=None, point_index=0, err=None, stream=None):
    """sde_josephson_run_fp64: one parameter point of Eq. 1 in FP64 on the GPU.
    x (absolute position in potential periods) and v are float64 CUDA tensors
    of one element per path; err: optional int32/uint32 CUDA tensor of one
    word, bit 1 set on a non-finite state."""
    p = JJPoint(point["gamma"], point["a"], point["omega"], point["f"], point["D"])
    _check(lib().sde_josephson_run_fp64(
        ctypes.byref(p), steps_per_period, x_in.numel(), total_steps, seed, point_index, n_begin, n_end,
        _ptr(x_in), _ptr(v_in), _ptr(vsum_in), _ptr(x_out), _ptr(v_out), _ptr(vsum_out), _ptr(err),
        _stream(stream)))


def debug_fail_allocation(nth):
    """sde_debug_fail_allocation: the nth allocation of the next create call fails."""
    lib().sde_debug_fail_allocation(nth)


def fp32_fma_probe(packed, iters, grid, block, sink, stream=None):
    """sde_fp32_fma_probe: launch the FP32 FMA throughput probe on `stream`;
    sink is a float32 CUDA tensor of at least grid * block elements.  Returns
    the FLOP the launch executes."""
    import torch
    assert sink.dtype == torch.float32 and sink.numel() >= grid * block
    flop = ctypes.c_double()
    _check(lib().sde_fp32_fma_probe(packed, iters, grid, block, _ptr(sink), ctypes.byref(flop), _stream(stream)))
    return flop.value


SURROGATE_BOX = ((0.0, 8.0), (1.0, 10.0), (0.0, 1.0), (0.5, 2.0), (-4.0, -1.0))  # a, omega, f, gamma, log10 D


class Mlp:
    """An sde_mlp: ensemble of surrogate networks with the library's own
    forward, backward and Adam kernels."""

    def __init__(self, n_in=5, hidden=256, n_hidden=3, members=4, max_batch=4096, lr=1e-3, beta1=0.9,
                 beta2=0.999, eps=1e-8, seed=0, box=SURROGATE_BOX):
        c = MlpConfig()
        c.n_in, c.hidden, c.n_hidden, c.n_members, c.max_batch = n_in, hidden, n_hidden, members, max_batch
        c.lr, c.beta1, c.beta2, c.eps, c.seed = lr, beta1, beta2, eps, seed
        for k, (lo, hi) in enumerate(box):
            c.lo[k], c.hi[k] = lo, hi
        h = _VP()
        _check(lib().sde_mlp_create(ctypes.byref(c), ctypes.byref(h)))
        self._h = h
        self.cfg = c
        self.members = members
        self.max_batch = max_batch
        self.n_params = lib().sde_mlp_num_params(h)

    def set_params(self, member, p, stream=None):
        _check(lib().sde_mlp_set_params(self._h, member, _ptr(p), _stream(stream)))

    def get_params(self, member, stream=None):
        import torch
        p = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _check(lib().sde_mlp_get_params(self._h, member, _ptr(p), _stream(stream)))
        return p

    def features(self, points_dev, stream=None):
        """points_dev: uint8 CUDA tensor holding n sde_jj_point records -> (n, 5) features."""
        import torch
        n = points_dev.numel() // ctypes.sizeof(JJPoint)
        X = torch.empty((n, 5), dtype=torch.float32, device="cuda")
        _check(lib().sde_mlp_features(self._h, _ptr(points_dev), n, _ptr(X), _stream(stream)))
        return X

    def forward(self, X, stream=None):
        """X: (B, n_in) float32 CUDA -> (mean, spread), each (B,)."""
        import torch
        B = X.shape[0]
        mean = torch.empty(B, dtype=torch.float32, device="cuda")
        spread = torch.empty(B, dtype=torch.float32, device="cuda")
        _check(lib().sde_mlp_forward(self._h, _ptr(X), B, _ptr(mean), _ptr(spread), _stream(stream)))
        return mean, spread

    def grad(self, member, X, y, stream=None):
        import torch
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(lib().sde_mlp_grad(self._h, member, _ptr(X), _ptr(y), X.shape[0], _ptr(g), _ptr(loss),
                                  _stream(stream)))
        return g, loss

    def set_lr(self, lr):
        _check(lib().sde_mlp_set_lr(self._h, lr))

    def use_tensor_cores(self, enable=True):
        """Tensor-core forward (default where the shape allows it) or the CUDA-core one."""
        _check(lib().sde_mlp_use_tensor_cores(self._h, 1 if enable else 0))

    def check(self):
        """Synchronise; raises SDEError (SDE_ERR_TIMEOUT) if a tensor-core forward
        kernel reported an expired wait since the last check."""
        _check(lib().sde_mlp_check(self._h))

    def train_step(self, X, y, loss=None, stream=None):
        _check(lib().sde_mlp_train_step(self._h, _ptr(X), _ptr(y), X.shape[0], _ptr(loss), _stream(stream)))

    def train_step_members(self, X, y, loss=None, stream=None):
        """X: (members, B, n_in), y: (members, B): one batch per member."""
        _check(lib().sde_mlp_train_step_members(self._h, _ptr(X), _ptr(y), X.shape[1], _ptr(loss),
                                                _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().sde_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def points_to_device(points):
    """Pack a list of parameter dicts into a CUDA uint8 tensor of sde_jj_point
    records (five doubles each: gamma, a, omega, f, D)."""
    import torch
    rec = np.array([(p["gamma"], p["a"], p["omega"], p["f"], p["D"]) for p in points], dtype=np.float64)
    rec = np.ascontiguousarray(rec.reshape(len(points), 5))
    assert rec.itemsize * 5 == ctypes.sizeof(JJPoint)
    return torch.from_numpy(rec.view(np.uint8).reshape(-1)).cuda()


def phase_histogram(phi, nbins, stream=None):
    """Counts of the phases phi (radians in [0, 2 pi)) in nbins equal bins."""
    import torch
    counts = torch.empty(nbins, dtype=torch.int64, device="cuda")
    _check(lib().sde_phase_histogram(_ptr(phi), phi.numel(), nbins, _ptr(counts), _stream(stream)))
    return counts
