"""Learned surrogate of the time-averaged velocity <<v>> of Eq. 1, with
simulator fallback (not in the paper; it builds on the batched sweep engine).

Pipeline, all compute in the CUDA library:
1. ``simulate``: <<v>> and its standard error for a list of parameter points,
   one persistent sweep launch (the engine of the batched Josephson sweep).
2. ``Surrogate.fit``: an ensemble of networks (5 -> 256 x 3 -> 1, SiLU) trained
   by the library's BF16 forward/backward/Adam kernels on simulated labels.
3. ``Surrogate.calibrate``: the ensemble spread times a factor k, chosen on
   held-out calibration points so that |prediction - label| <= k spread for a
   given share of them, is the predicted error.
4. ``Surrogate.answer``: network prediction where the predicted error is at
   most the tolerance, the simulator's own <<v>> elsewhere (fallback).

The per-point arithmetic (features, the networks and their spread, the
simulations) runs in the CUDA library; this module batches and shuffles, and
takes the scalar control decisions on the host (the step-size schedule, the
calibration quantile, the fallback mask).
"""
import time

import numpy as np
import torch

from . import sde

STEPS_PER_PERIOD = 200


def simulate(points, paths, steps, seed, stream=None, init_seed=None):
    """<<v>> (mean over paths of the window average, last half of the run) and
    its standard error for every point; returns (mean, se, seconds) as numpy."""
    n = len(points)
    pa = np.full(n, paths, dtype=np.int64)
    st = np.full(n, steps, dtype=np.int64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ens = sde.Ensemble.josephson(points, pa, st, seed, steps_per_period=STEPS_PER_PERIOD)
    total = n * paths
    g = torch.Generator(device="cuda")
    g.manual_seed(seed if init_seed is None else init_seed)
    x0 = torch.rand(total, device="cuda", generator=g)
    v0 = torch.rand(total, device="cuda", generator=g) * 4.0 - 2.0
    w = torch.empty(total, dtype=torch.int32, device="cuda")
    vs = torch.empty(total, dtype=torch.float64, device="cuda")
    ens.run_josephson(0, steps, x0, v0, x0, v0, w, vs, stream=stream)
    obs = ens.observables()
    dt = time.perf_counter() - t0
    simulate.last_kernel_ms = ens.last_kernel_ms()
    ens.close()
    return obs["mean"].copy(), obs["se"].copy(), dt


class Surrogate:
    def __init__(self, members=4, max_batch=16384, lr=1e-3, seed=0):
        self.mlp = sde.Mlp(members=members, max_batch=max_batch, lr=lr, seed=seed)
        self.max_batch = max_batch
        self.lr = lr
        self.k = None

    def features(self, points):
        return self.mlp.features(sde.points_to_device(points))

    def fit(self, points, y, epochs=60, batch=1024, seed=0, lr_final=1e-5):
        """Train every member on its own bootstrap resample of (features(points),
        y) -- the spread of such an ensemble tracks its error; returns the
        last losses."""
        X = self.features(points)
        yd = torch.as_tensor(np.asarray(y, dtype=np.float32)).cuda()
        n = X.shape[0]
        M = self.mlp.members
        rng = np.random.default_rng(seed)
        boot = [rng.integers(0, n, n) for _ in range(M)]
        loss = torch.zeros(M, device="cuda")
        steps = epochs * max(1, n // batch)
        k = 0
        for ep in range(epochs):
            order = [b[rng.permutation(n)] for b in boot]
            for b0 in range(0, n - batch + 1, batch):
                # cosine decay of the step size from lr to lr_final
                self.mlp.set_lr(lr_final + 0.5 * (self.lr - lr_final) * (1 + np.cos(np.pi * k / steps)))
                idx = torch.from_numpy(np.concatenate([o[b0:b0 + batch] for o in order])).cuda()
                self.mlp.train_step_members(X[idx].view(M, batch, -1).contiguous(),
                                            yd[idx].view(M, batch).contiguous(), loss)
                k += 1
        return loss.cpu().numpy()

    def predict(self, points):
        """(mean, spread) numpy arrays of the ensemble."""
        X = self.features(points)
        means, spreads = [], []
        for b0 in range(0, X.shape[0], self.max_batch):
            m, s = self.mlp.forward(X[b0:b0 + self.max_batch].contiguous())
            means.append(m)
            spreads.append(s)
        return torch.cat(means).cpu().numpy(), torch.cat(spreads).cpu().numpy()

    def calibrate(self, points, y, coverage=0.95, bins=8):
        """Factors k with |prediction - y| <= k spread on `coverage` of the
        calibration points, one per bin of spread (quantile bins), so that the
        predicted error k(spread) spread adapts to regions where the spread is
        more or less faithful.  Returns the overall factor."""
        mean, spread = self.predict(points)
        ratio = np.abs(mean - np.asarray(y)) / np.maximum(spread, 1e-12)
        self.edges = np.quantile(spread, np.linspace(0, 1, bins + 1)[1:-1])
        which = np.searchsorted(self.edges, spread)
        self.kbin = np.array([np.quantile(ratio[which == b], coverage) if np.any(which == b)
                              else np.quantile(ratio, coverage) for b in range(bins)])
        self.k = float(np.quantile(ratio, coverage))
        return self.k

    def predicted_error(self, spread):
        return self.kbin[np.searchsorted(self.edges, spread)] * spread

    def answer(self, points, tol, fallback_paths, steps, seed):
        """Network prediction where its predicted error is <= tol, simulator elsewhere.
        Returns dict(value, predicted_error, fallback mask, seconds split)."""
        assert self.k is not None, "calibrate first"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mean, spread = self.predict(points)
        t_mlp = time.perf_counter() - t0
        perr = self.predicted_error(spread)
        fb = perr > tol
        value = mean.astype(np.float64).copy()
        t_sim = 0.0
        if fb.any():
            sel = [points[i] for i in np.flatnonzero(fb)]
            vm, vse, t_sim = simulate(sel, fallback_paths, steps, seed)
            value[fb] = vm
            perr = perr.astype(np.float64)
            perr[fb] = vse
        return dict(value=value, predicted_error=perr, fallback=fb, t_mlp=t_mlp, t_sim=t_sim)
