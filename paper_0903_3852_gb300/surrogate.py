"""Learned surrogate of the time-averaged velocity <<v>> of Eq. 1, with
simulator fallback (not in the paper; it builds on the batched sweep engine).

Pipeline, all compute in the CUDA library:
1. ``simulate``: <<v>> and its standard error for a list of parameter points,
   one persistent sweep launch (the engine of the batched Josephson sweep).
2. ``Surrogate.fit``: an ensemble of networks (5 -> 256 x 3 -> 1, SiLU) trained
   by the library's BF16 forward/backward/Adam kernels on simulated labels.
3. ``Surrogate.fit_error_model``: a second network (the same kernels) learns
   log |prediction - label| on held-out points from the parameters, the
   ensemble's prediction and its spread: the ensemble spread alone misses the
   errors the members share (the members agree on the smooth edge of a
   phase-locked plateau of <<v>> = 0, for instance).
   ``Surrogate.calibrate``: selective calibration on further held-out points.
   The network is trusted below a threshold on the error model's prediction,
   the largest for which the calibration points below it miss the tolerance
   (beyond their own labels' noise) at a rate of at most `risk`, counted
   conservatively ((misses + 1) / (points + 1)); the predicted error is tol
   times the error model's prediction over the threshold.
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
        # error model: inputs = the 5 parameter features, the ensemble mean and
        # its log spread; output = log |mean - <<v>>|
        self.err_mlp = sde.Mlp(n_in=7, members=2, max_batch=max_batch, lr=lr, seed=seed + 101)
        self.max_batch = max_batch
        self.lr = lr
        self.tau = None

    def features(self, points):
        return self.mlp.features(sde.points_to_device(points))

    def fit(self, points, y, epochs=60, batch=1024, seed=0, lr_final=1e-5):
        """Train every member on its own bootstrap resample of (features(points),
        y) -- the spread of such an ensemble tracks its error; returns the
        last losses."""
        return self._fit(self.mlp, self.features(points), y, epochs, batch, seed, lr_final)

    def _fit(self, mlp, X, y, epochs, batch, seed, lr_final):
        yd = torch.as_tensor(np.asarray(y, dtype=np.float32)).cuda()
        n = X.shape[0]
        M = mlp.members
        rng = np.random.default_rng(seed)
        boot = [rng.integers(0, n, n) for _ in range(M)]
        loss = torch.zeros(M, device="cuda")
        steps = epochs * max(1, n // batch)
        k = 0
        for ep in range(epochs):
            order = [b[rng.permutation(n)] for b in boot]
            for b0 in range(0, n - batch + 1, batch):
                # cosine decay of the step size from lr to lr_final
                mlp.set_lr(lr_final + 0.5 * (self.lr - lr_final) * (1 + np.cos(np.pi * k / steps)))
                idx = torch.from_numpy(np.concatenate([o[b0:b0 + batch] for o in order])).cuda()
                mlp.train_step_members(X[idx].view(M, batch, -1).contiguous(),
                                       yd[idx].view(M, batch).contiguous(), loss)
                k += 1
        return loss.cpu().numpy()

    def _predict_dev(self, X):
        means, spreads = [], []
        for b0 in range(0, X.shape[0], self.max_batch):
            m, s = self.mlp.forward(X[b0:b0 + self.max_batch].contiguous())
            means.append(m)
            spreads.append(s)
        return torch.cat(means), torch.cat(spreads)

    def predict(self, points):
        """(mean, spread) numpy arrays of the ensemble."""
        m, s = self._predict_dev(self.features(points))
        return m.cpu().numpy(), s.cpu().numpy()

    def _error_inputs(self, X, mean, spread):
        # the 5 features, the prediction and log10 of the spread, all O(1)
        return torch.cat([X, mean[:, None], (torch.log10(spread.clamp_min(1e-7)) + 3.0)[:, None] / 2.0],
                         dim=1).contiguous()

    def _log_error_dev(self, X, mean, spread):
        E = self._error_inputs(X, mean, spread)
        out = []
        for b0 in range(0, E.shape[0], self.max_batch):
            out.append(self.err_mlp.forward(E[b0:b0 + self.max_batch].contiguous())[0])
        return torch.cat(out)

    def fit_error_model(self, points, y, epochs=200, batch=1024, seed=1, lr_final=1e-5):
        """Train the error model on held-out points: target log(|mean - y| + 1e-4)."""
        X = self.features(points)
        mean, spread = self._predict_dev(X)
        r = np.abs(mean.cpu().numpy().astype(np.float64) - np.asarray(y, dtype=np.float64))
        target = np.log(r + 1e-4)
        return self._fit(self.err_mlp, self._error_inputs(X, mean, spread), target, epochs, batch, seed, lr_final)

    def predict_with_error(self, points):
        """(mean, spread, error-model log error) numpy arrays."""
        X = self.features(points)
        mean, spread = self._predict_dev(X)
        le = self._log_error_dev(X, mean, spread)
        return mean.cpu().numpy(), spread.cpu().numpy(), le.cpu().numpy()

    def calibrate(self, points, y, se, tol, risk=5e-4):
        """Threshold tau on the error model's log error, on held-out calibration
        points with labels y of standard error se: a point counts as a miss when
        |prediction - y| > tol + 3 se, i.e. when the label rules out an error
        within tol (the acceptance rule of the evaluation, against its own
        reference); tau is the largest score at which the points scoring <= tau
        have (misses + 1) / (points + 1) <= risk.  Returns (tau, share of the
        calibration points answered)."""
        mean, spread, le = self.predict_with_error(points)
        y, se = np.asarray(y, dtype=np.float64), np.asarray(se, dtype=np.float64)
        miss = ~(np.abs(mean - y) <= tol + 3.0 * se)  # NaN counts as a miss
        le = np.where(np.isfinite(le), le, np.inf)
        order = np.argsort(le, kind="stable")
        misses = np.cumsum(miss[order])
        count = np.arange(1, len(order) + 1)
        ok = ((misses + 1.0) / (count + 1.0) <= risk) & np.isfinite(le[order])
        self.tau = float(le[order][np.flatnonzero(ok)[-1]]) if ok.any() else -np.inf
        self.tol = tol
        return self.tau, float(np.mean(le <= self.tau))

    def predicted_error(self, log_error):
        """tol x exp(log error - tau): at most tol exactly where the network answers."""
        with np.errstate(over="ignore"):
            return self.tol * np.exp(np.asarray(log_error, dtype=np.float64) - self.tau)

    def answer(self, points, tol, fallback_paths, steps, seed):
        """Network prediction where its predicted error is <= tol, simulator elsewhere.
        Returns dict(value, predicted_error, fallback mask, seconds split)."""
        assert self.tau is not None, "calibrate first"
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mean, spread, le = self.predict_with_error(points)
        t_mlp = time.perf_counter() - t0
        perr = self.predicted_error(le)
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
