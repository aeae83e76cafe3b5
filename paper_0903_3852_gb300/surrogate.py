"""Learned surrogate of the time-averaged velocity <<v>> of Eq. 1, with
simulator fallback (not in the paper; it builds on the batched sweep engine).

Pipeline, all compute in the CUDA library:
1. ``simulate``: <<v>> and its standard error for a list of parameter points,
   one persistent sweep launch (the engine of the batched Josephson sweep).
2. ``Surrogate.fit``: an ensemble of networks (5 -> 256 x 3 -> 1, SiLU) trained
   by the library's BF16 forward/backward/Adam kernels on simulated labels.
3. ``Surrogate.calibrate``: selective calibration on held-out points.  The
   network is trusted below a spread threshold tau, the largest for which the
   calibration points with spread <= tau miss the tolerance (beyond their own
   labels' noise) at a rate of at most `risk`, counted conservatively
   ((misses + 1) / (points + 1)); the predicted error is tol * spread / tau.
4. ``Surrogate.answer``: network prediction where the predicted error is at
   most the tolerance, the simulator's own <<v>> elsewhere (fallback; also
   wherever the prediction is not finite).

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
    def __init__(self, members=4, max_batch=131072, lr=1e-3, seed=0):
        self.mlp = sde.Mlp(members=members, max_batch=max_batch, lr=lr, seed=seed)
        self.max_batch = max_batch
        self.lr = lr
        self.tau = None

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

    def calibrate(self, points, y, se, tol, risk=5e-4):
        """Spread threshold tau on held-out calibration points with labels y of
        standard error se: a point counts as a miss when |prediction - y| >
        tol + 3 se, i.e. when the label rules out an error within tol (the
        acceptance rule of the evaluation, against its own reference); tau is
        the largest spread at which the points with spread <= tau have
        (misses + 1) / (points + 1) <= risk.  Returns (tau, share of the
        calibration points answered)."""
        mean, spread = self.predict(points)
        y, se = np.asarray(y, dtype=np.float64), np.asarray(se, dtype=np.float64)
        miss = ~(np.abs(mean - y) <= tol + 3.0 * se)  # NaN counts as a miss
        order = np.argsort(spread, kind="stable")
        misses = np.cumsum(miss[order])
        count = np.arange(1, len(order) + 1)
        ok = (misses + 1.0) / (count + 1.0) <= risk
        self.tau = float(spread[order][np.flatnonzero(ok)[-1]]) if ok.any() else 0.0
        self.tol = tol
        return self.tau, float(np.mean(spread <= self.tau)) if self.tau > 0 else 0.0

    def predicted_error(self, spread):
        if self.tau <= 0.0:
            return np.full(np.shape(spread), np.inf)
        return self.tol * np.asarray(spread, dtype=np.float64) / self.tau

    def answer(self, points, tol, fallback_paths, steps, seed):
        """Network prediction where its predicted error is <= tol, simulator elsewhere.
        Returns dict(value, predicted_error, fallback mask, seconds split)."""
        assert self.tau is not None, "calibrate first"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mean, spread = self.predict(points)
        t_mlp = time.perf_counter() - t0
        perr = self.predicted_error(spread)
        fb = ~(perr <= tol) | ~np.isfinite(mean)
        value = mean.astype(np.float64).copy()
        t_sim = 0.0
        if fb.any():
            sel = [points[i] for i in np.flatnonzero(fb)]
            vm, vse, t_sim = simulate(sel, fallback_paths, steps, seed)
            value[fb] = vm
            perr = perr.astype(np.float64)
            perr[fb] = vse
        return dict(value=value, predicted_error=perr, fallback=fb, t_mlp=t_mlp, t_sim=t_sim)
