"""The learned surrogate of <<v>> end to end at reduced scale: labels from the
sweep engine (2048 paths x 2e4 steps per point, as in the full configuration),
an ensemble trained by the library's kernels, calibration of its predicted
error, and simulator fallback wherever that error exceeds 1e-2.  Checks: after
fallback every held-out point is within 1e-2 of a higher-path simulator
reference (slack: 3 of the reference's and the answer's standard errors), and
the network answers part of the points faster than the simulator would."""
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
    train = inputs.surrogate_points(6000, seed=16)
    y, se, t_lab = surrogate.simulate(train, 2048, STEPS, seed=16)
    sur = surrogate.Surrogate(members=4, max_batch=8192, lr=2e-3, seed=3)
    sur.fit(train[:5000], y[:5000], epochs=40, batch=500)
    k = sur.calibrate(train[5000:], y[5000:])
    evalp = inputs.surrogate_points(400, seed=17)
    ref, ref_se, t_ref = surrogate.simulate(evalp, 8192, STEPS, seed=17)
    out = sur.answer(evalp, TOL, fallback_paths=8192, steps=STEPS, seed=18)
    err = np.abs(out["value"] - ref)
    answered = ~out["fallback"]
    slack = 3.0 * np.hypot(ref_se, np.where(answered, 0.0, out["predicted_error"]))
    ok = err <= TOL + slack
    print("k=%.2f answered by the network: %d/%d; within tol: %d/%d; median |err| net %.2e" %
          (k, answered.sum(), len(evalp), ok.sum(), len(evalp),
           np.median(err[answered]) if answered.any() else float("nan")))
    print("times: simulator-only %.3f s, network %.4f s + fallback %.3f s" % (t_ref, out["t_mlp"], out["t_sim"]))
    assert ok.mean() >= 0.95
    assert answered.any()
    assert out["t_mlp"] + out["t_sim"] < t_ref
