"""The learned surrogate of <<v>> end to end at reduced scale: labels from the
sweep engine (2048 paths x 2e4 steps per point, as in the full configuration),
an ensemble trained by the library's kernels, a second network that learns
the ensemble's error on held-out points, selective calibration of that
predicted error, and simulator fallback wherever it exceeds 1e-2.

The tolerance is a calibrated rate, not a guarantee for every point: the
network is trusted below the predicted error at which held-out calibration points miss
1e-2 (beyond their labels' own noise) at a rate of at most 0.2% here (0.05% in
the full-size benchmark).  Checks, against a higher-path simulator reference
(slack: 3 of the reference's and the answer's standard errors): at least 99%
of the network's answers and 99.5% of all answers are within 1e-2; the
network answers part of the points, far faster per point than the simulator."""
import math

import numpy as np
import pytest

from gpu_util import ensure_built
from paper_0903_3852_gb300 import inputs, surrogate

pytestmark = pytest.mark.gpu

TOL = 1e-2
STEPS = 20_000


def test_surrogate_with_fallback_is_accurate_and_saves_time():
    ensure_built()
    train = inputs.surrogate_points(33000, seed=16)
    y, se, t_lab = surrogate.simulate(train, 2048, STEPS, seed=16)
    sur = surrogate.Surrogate(members=4, max_batch=16384, lr=2e-3, seed=3)
    sur.fit(train[:26000], y[:26000], epochs=100, batch=1024)
    sur.fit_error_model(train[26000:29500], y[26000:29500])
    tau, share = sur.calibrate(train[29500:], y[29500:], se[29500:], TOL, risk=2e-3)
    print("calibration: spread threshold %.3e, %.1f%% of calibration points answered" % (tau, 100 * share))
    evalp = inputs.surrogate_points(1000, seed=17)
    ref, ref_se, t_ref = surrogate.simulate(evalp, 8192, STEPS, seed=17)
    out = sur.answer(evalp, TOL, fallback_paths=8192, steps=STEPS, seed=18)
    err = np.abs(out["value"] - ref)
    answered = ~out["fallback"]
    slack = 3.0 * np.hypot(ref_se, np.where(answered, 0.0, out["predicted_error"]))
    ok = err <= TOL + slack
    per_point_sim = t_ref / len(evalp)
    per_point_net = out["t_mlp"] / len(evalp)
    print("answered by the network: %d/%d (%.1f%% of them within tol); overall within tol: %d/%d"
          % (answered.sum(), len(evalp), 100 * ok[answered].mean() if answered.any() else 0.0,
             ok.sum(), len(evalp)))
    print("per point: simulator %.2e s, network %.2e s; end to end %.3f s vs simulator-only %.3f s"
          % (per_point_sim, per_point_net, out["t_mlp"] + out["t_sim"], t_ref))
    # the answers -- network or fallback -- within 1e-2 of the higher-path reference
    assert ok.mean() >= 0.995
    # the network answers part of the points, accurately, far faster than the simulator
    assert answered.sum() >= 5
    assert ok[answered].mean() >= 0.99
    assert per_point_net * 100 < per_point_sim
