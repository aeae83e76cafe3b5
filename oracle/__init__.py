"""FP64 CPU oracle for ensemble SDE integration (Januszewski & Kostur, arXiv:0903.3852).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code with
the CUDA library.  The C core lives in sde_oracle.c (Philox4x32-10, Box-Muller,
SRK2 of Alg. 2 for Eq. 1 and Eq. 2, the direct and the Eq. 3 mean-field coupling
sums, the order parameter); mlp.py holds the FP64 reference of the surrogate
network.  Each function cites the passage it follows.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_f64p = ctypes.POINTER(ctypes.c_double)


class JJParams(ctypes.Structure):
    """Parameters of Eq. 1: friction gamma, drive amplitude a, drive frequency
    omega, bias f and noise intensity D (k_B T)."""
    _fields_ = [("gamma", ctypes.c_double), ("a", ctypes.c_double),
                ("omega", ctypes.c_double), ("f", ctypes.c_double),
                ("D", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.oracle_philox4x32_rounds.argtypes = [_u32p, _u32p, ctypes.c_int, _u32p]
        L.oracle_uniform.argtypes = [ctypes.c_uint32]
        L.oracle_uniform.restype = ctypes.c_double
        L.oracle_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _f64p, _f64p]
        L.oracle_gaussian.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, ctypes.c_uint64]
        L.oracle_gaussian.restype = ctypes.c_double
        L.oracle_jj_step.argtypes = [_f64p, _f64p, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.POINTER(JJParams), ctypes.c_double]
        L.oracle_jj_rhs.argtypes = [ctypes.c_double, _f64p, ctypes.POINTER(JJParams), _f64p]
        L.oracle_jj_run.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p,
                                    ctypes.POINTER(JJParams), ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                    ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.oracle_jj_euler_step.argtypes = [_f64p, _f64p, ctypes.c_uint64, ctypes.c_double,
                                           ctypes.POINTER(JJParams), ctypes.c_double]
        L.oracle_jj_run_scheme.argtypes = L.oracle_jj_run.argtypes + [ctypes.c_int]
        L.oracle_linear_step.argtypes = [_f64p, _f64p] + [ctypes.c_double] * 6
        L.oracle_linear_euler_step.argtypes = [_f64p, _f64p] + [ctypes.c_double] * 6
        L.oracle_kuramoto_coupling_direct.argtypes = [ctypes.c_int64, _f64p, _f64p,
                                                      ctypes.c_double, _f64p]
        L.oracle_kuramoto_coupling_meanfield.argtypes = [ctypes.c_int64, _f64p,
                                                         ctypes.c_double, _f64p]
        L.oracle_order_parameter.argtypes = [ctypes.c_int64, _f64p]
        L.oracle_order_parameter.restype = ctypes.c_double
        L.oracle_kuramoto_run.argtypes = [ctypes.c_int64, _f64p, _f64p, _f64p,
                                          ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_uint32, _f64p,
                                          ctypes.c_int64]
        L.oracle_kuramoto_run_scheme.argtypes = L.oracle_kuramoto_run.argtypes + [ctypes.c_int]
        _lib = L
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


TAG_JOSEPHSON = 1
TAG_KURAMOTO = 2


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC'11) on a batch of counters.
    ctr: (n, 4) uint32, key: (2,) uint32 -> (n, 4) uint32."""
    L = lib()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    kp = key.ctypes.data_as(_u32p)
    for i in range(ctr.shape[0]):
        L.oracle_philox4x32_10(ctr[i].ctypes.data_as(_u32p), kp, out[i].ctypes.data_as(_u32p))
    return out


def philox4x32_rounds(ctr, key, rounds):
    """The first `rounds` rounds of Philox4x32 (SC'11, Sec. 4): one counter
    (4,) uint32 and key (2,) uint32 -> (4,) uint32.  rounds = 10 equals
    philox4x32_10; fewer rounds expose the round function and the key
    schedule to tests."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty(4, dtype=np.uint32)
    lib().oracle_philox4x32_rounds(ctr.ctypes.data_as(_u32p), key.ctypes.data_as(_u32p), int(rounds),
                                   out.ctypes.data_as(_u32p))
    return out


def seed_key(seed):
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def uniform(w):
    return lib().oracle_uniform(int(w))


def box_muller(w0, w1):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().oracle_box_muller(int(w0), int(w1), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def gaussian(seed, tag, c1, c2, n):
    """The standard Gaussian used by step n of noise stream (c1, c2, tag)."""
    return lib().oracle_gaussian(seed, tag, c1, c2, n)


def jj_params(gamma, a, omega, f, D):
    return JJParams(gamma, a, omega, f, D)


def jj_step(x, v, n, dt, p, psi):
    """One SRK2 step (Alg. 2) of Eq. 1 with a given Gaussian psi -> (x, v)."""
    xc, vc = ctypes.c_double(x), ctypes.c_double(v)
    lib().oracle_jj_step(ctypes.byref(xc), ctypes.byref(vc), n, dt, ctypes.byref(p), psi)
    return xc.value, vc.value


def jj_euler_step(x, v, n, dt, p, psi):
    """One Euler-Maruyama step of Eq. 1 (the first-order scheme of PROG2) -> (x, v)."""
    xc, vc = ctypes.c_double(x), ctypes.c_double(v)
    lib().oracle_jj_euler_step(ctypes.byref(xc), ctypes.byref(vc), n, dt, ctypes.byref(p), psi)
    return xc.value, vc.value


def jj_rhs(t, y, p):
    y, yp = _f64(y)
    dy = np.empty(2)
    lib().oracle_jj_rhs(t, yp, ctypes.byref(p), dy.ctypes.data_as(_f64p))
    return dy


SCHEME_SRK2, SCHEME_EULER = 0, 1


def jj_run(x, v, p, steps_per_period, n_begin, n_end, total_steps, seed, point=0,
           path0=0, vsum=None, scheme=SCHEME_SRK2):
    """Advance a batch of Eq. 1 paths (Alg. 1 with Alg. 2, or Euler-Maruyama
    for scheme=SCHEME_EULER); returns (x, v, vsum)."""
    x, xp = _f64(np.array(x, dtype=np.float64, copy=True))
    v, vp = _f64(np.array(v, dtype=np.float64, copy=True))
    vs = np.zeros_like(x) if vsum is None else np.array(vsum, dtype=np.float64, copy=True)
    vs, vsp = _f64(vs)
    lib().oracle_jj_run_scheme(x.size, xp, vp, vsp, ctypes.byref(p), steps_per_period,
                               n_begin, n_end, total_steps, seed, point, path0, scheme)
    return x, v, vs


def linear_step(x, v, dt, gamma, kappa, f, D, psi):
    xc, vc = ctypes.c_double(x), ctypes.c_double(v)
    lib().oracle_linear_step(ctypes.byref(xc), ctypes.byref(vc), dt, gamma, kappa, f, D, psi)
    return xc.value, vc.value


def linear_euler_step(x, v, dt, gamma, kappa, f, D, psi):
    xc, vc = ctypes.c_double(x), ctypes.c_double(v)
    lib().oracle_linear_euler_step(ctypes.byref(xc), ctypes.byref(vc), dt, gamma, kappa, f, D, psi)
    return xc.value, vc.value


def coupling_direct(phi, Kmat=None, Kconst=0.0):
    phi, pp = _f64(phi)
    out = np.empty_like(phi)
    if Kmat is None:
        lib().oracle_kuramoto_coupling_direct(phi.size, pp, None, Kconst, out.ctypes.data_as(_f64p))
    else:
        K, kp = _f64(Kmat)
        assert K.shape == (phi.size, phi.size)
        lib().oracle_kuramoto_coupling_direct(phi.size, pp, kp, Kconst, out.ctypes.data_as(_f64p))
    return out


def coupling_meanfield(phi, Kconst):
    phi, pp = _f64(phi)
    out = np.empty_like(phi)
    lib().oracle_kuramoto_coupling_meanfield(phi.size, pp, Kconst, out.ctypes.data_as(_f64p))
    return out


def order_parameter(phi):
    phi, pp = _f64(phi)
    return lib().oracle_order_parameter(phi.size, pp)


def kuramoto_run(phi, omega, D, dt, n_begin, n_end, seed, replica, Kmat=None, Kconst=0.0,
                 meanfield=False, sample_every=0, scheme=SCHEME_SRK2):
    """Advance one replica of Eq. 2 by SRK2 (or Euler-Maruyama for
    scheme=SCHEME_EULER); returns (phi, r samples or None)."""
    phi, pp = _f64(np.array(phi, dtype=np.float64, copy=True))
    om, op = _f64(omega)
    kp = None
    if Kmat is not None:
        K, kp = _f64(Kmat)
    r = None
    rp = None
    if sample_every > 0:
        ns = -(-(n_end - n_begin) // sample_every)
        r = np.zeros(ns + 1)
        rp = r.ctypes.data_as(_f64p)
    lib().oracle_kuramoto_run_scheme(phi.size, pp, op, kp, Kconst, 1 if meanfield else 0, D, dt,
                                     n_begin, n_end, seed, replica, rp, sample_every, scheme)
    return phi, r
