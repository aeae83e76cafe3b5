"""Seeded synthetic inputs for the ensemble-SDE workloads.

This module holds none of the method's arithmetic: it only draws initial
states, parameter grids and coupling matrices with numpy's seeded generator, so
that the CUDA path and the FP64 oracle start from identical inputs.  The noise
of the method itself is drawn inside each side by its own Philox4x32-10.

Workloads (sizes as used by the tests and the benchmark):

- ``josephson_plain``: Eq. 1 at the parameters of the paper's Fig. 2 regime
  (gamma 0.9, a 4.2, omega 4.9, f 0.1, D 1e-3), 1024 paths, dt = (2 pi /
  omega) / 200, 20,000 steps (100 drive periods); x0 ~ U[0, 1),
  v0 ~ U[-2, 2); noise seed 0.
- ``josephson_sweep``: 512 parameter points, f on 171 values in [0, 0.5]
  times D in {1e-4, 1e-3, 1e-2}, D-major, the first 512 of the 513 pairs;
  a 4.2, omega 4.9, gamma 0.9; paths per point log-uniform in [256, 8192],
  steps per point log-uniform in [1e4, 1e5]; all drawn from seed 1.
- ``kuramoto_uniform``: Eq. 2 with K_ij = K / N, N 4096, 64 replicas,
  omega_i ~ N(0, 1) independently per replica, K 2, D 0.05, phi0 ~ U[0, 2 pi),
  dt 0.01, 10^4 steps, samples of r every 100 steps.
- ``kuramoto_general``: N 8192, 256 replicas, K_ij = (K0 / N)(1 + 0.5 u_ij),
  u_ij ~ U[-1, 1], K0 3, D 0.02, dt 0.005, 5000 steps.
- ``josephson_fig2``: the Fig. 2 ensemble, 2^19 paths at the parameters above,
  dt = (2 pi / omega) / 100, 2 10^5 steps.
- ``kuramoto_fig4``: the Fig. 4 ensemble, one replica of 2^24 oscillators,
  omega_i = 0, K 4, D 1, dt 0.01, 2000 steps, samples every 100.
"""
import math

import numpy as np

TWO_PI = 2.0 * math.pi


def josephson_plain(paths=1024, steps=20_000, seed=0):
    rng = np.random.default_rng(seed)
    x0 = rng.random(paths).astype(np.float32)
    v0 = rng.uniform(-2.0, 2.0, paths).astype(np.float32)
    return dict(
        points=[dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)],
        paths=np.array([paths], dtype=np.int64),
        steps=np.array([steps], dtype=np.int64),
        steps_per_period=200,
        seed=seed,
        x0=x0,
        v0=v0,
    )


def josephson_fig2(paths=2 ** 19, periods=2000, steps_per_period=100, seed=0):
    """The ensemble of the paper's Fig. 2: 524,288 paths of Eq. 1 at a = 4.2,
    gamma = 0.9, omega = 4.9, D = 0.001, f = 0.1, dt = 0.01 (2 pi / omega),
    t in (0, 2000 (2 pi / omega)): 2e5 steps."""
    rng = np.random.default_rng(seed)
    steps = periods * steps_per_period
    return dict(points=[dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)],
                paths=np.array([paths], dtype=np.int64), steps=np.array([steps], dtype=np.int64),
                steps_per_period=steps_per_period, seed=seed,
                x0=rng.random(paths).astype(np.float32),
                v0=rng.uniform(-2.0, 2.0, paths).astype(np.float32))


def sweep_grid(n_points=512, n_f=171, D_values=(1e-4, 1e-3, 1e-2)):
    f = np.linspace(0.0, 0.5, n_f)
    pts = [dict(gamma=0.9, a=4.2, omega=4.9, f=float(fv), D=float(Dv))
           for Dv in D_values for fv in f]
    return pts[:n_points]


def log_uniform_int(rng, lo, hi, n):
    return np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), n))).astype(np.int64)


def josephson_sweep(n_points=512, path_range=(256, 8192), step_range=(10_000, 100_000),
                    seed=1, steps_per_period=200):
    rng = np.random.default_rng(seed)
    pts = sweep_grid(n_points)
    paths = log_uniform_int(rng, *path_range, n_points)
    steps = log_uniform_int(rng, *step_range, n_points)
    total = int(paths.sum())
    x0 = rng.random(total).astype(np.float32)
    v0 = rng.uniform(-2.0, 2.0, total).astype(np.float32)
    return dict(points=pts, paths=paths, steps=steps, steps_per_period=steps_per_period,
                seed=seed, x0=x0, v0=v0)


def josephson_custom(points, paths, steps, seed, steps_per_period=200, init_seed=None):
    """Arbitrary list of parameter points with per-point path and step counts."""
    rng = np.random.default_rng(seed if init_seed is None else init_seed)
    paths = np.asarray(paths, dtype=np.int64)
    steps = np.asarray(steps, dtype=np.int64)
    total = int(paths.sum())
    x0 = rng.random(total).astype(np.float32)
    v0 = rng.uniform(-2.0, 2.0, total).astype(np.float32)
    return dict(points=list(points), paths=paths, steps=steps,
                steps_per_period=steps_per_period, seed=seed, x0=x0, v0=v0)


def kuramoto_uniform(n_osc=4096, replicas=64, K=2.0, D=0.05, dt=0.01, steps=10_000,
                     sample_every=100, seed=0):
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((replicas, n_osc)).astype(np.float32)
    phi0 = rng.uniform(0.0, TWO_PI, (replicas, n_osc)).astype(np.float32)
    return dict(n_osc=n_osc, replicas=replicas, K=K, D=D, dt=dt, steps=steps,
                sample_every=sample_every, seed=seed, omega=omega, phi0=phi0)


def kuramoto_general(n_osc=8192, replicas=256, K0=3.0, D=0.02, dt=0.005, steps=5000,
                     sample_every=100, seed=0):
    """K_ij = (K0 / N)(1 + 0.5 u_ij), row i = receiving oscillator, float32."""
    rng = np.random.default_rng(seed)
    omega = rng.standard_normal((replicas, n_osc)).astype(np.float32)
    phi0 = rng.uniform(0.0, TWO_PI, (replicas, n_osc)).astype(np.float32)
    u = rng.random((n_osc, n_osc), dtype=np.float32)
    u *= 2.0
    u -= 1.0
    Kmat = u
    Kmat *= np.float32(0.5)
    Kmat += np.float32(1.0)
    Kmat *= np.float32(K0 / n_osc)
    return dict(n_osc=n_osc, replicas=replicas, K0=K0, D=D, dt=dt, steps=steps,
                sample_every=sample_every, seed=seed, omega=omega, phi0=phi0, Kmat=Kmat)


def kuramoto_fig4(n_osc=2 ** 24, K=4.0, D=1.0, dt=0.01, steps=2000, sample_every=100, seed=0):
    """The ensemble of the paper's Fig. 4: one replica of 2^24 identical
    oscillators (omega_i = 0), K = 4, T = 1, phases uniform on [0, 2 pi)."""
    rng = np.random.default_rng(seed)
    phi0 = rng.uniform(0.0, TWO_PI, (1, n_osc)).astype(np.float32)
    omega = np.zeros((1, n_osc), dtype=np.float32)
    return dict(n_osc=n_osc, replicas=1, K=K, D=D, dt=dt, steps=steps, sample_every=sample_every,
                seed=seed, omega=omega, phi0=phi0)


SURROGATE_BOX = dict(a=(0.0, 8.0), omega=(1.0, 10.0), f=(0.0, 1.0), gamma=(0.5, 2.0),
                     log10D=(-4.0, -1.0))


def surrogate_points(n, seed):
    """Parameter points uniform in the surrogate's box (log10 D uniform)."""
    rng = np.random.default_rng(seed)
    cols = {k: rng.uniform(lo, hi, n) for k, (lo, hi) in SURROGATE_BOX.items()}
    return [dict(gamma=float(cols["gamma"][i]), a=float(cols["a"][i]),
                 omega=float(cols["omega"][i]), f=float(cols["f"][i]),
                 D=float(10.0 ** cols["log10D"][i])) for i in range(n)]
