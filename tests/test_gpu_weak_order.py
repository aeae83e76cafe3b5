"""Weak order of the GPU integrators on Eq. 1, by Richardson differences.

<v> (the window average of v over the second half of 40 drive periods, a whole
number of periods, so the discrete average adds no quadrature error) is
measured with 2^23 paths per point at dt = T/P for P = 25, 50, 100 (SRK2,
Alg. 2) and P = 100, 200, 400 (Euler-Maruyama, PROG2's first-order scheme,
Sec. 4.2).  For a scheme of weak order p the successive differences
<v>_P - <v>_2P shrink by 2^p per halving of dt: about 2 for Euler-Maruyama;
SRK2, a second-order scheme, must shrink them by clearly more than 2 (at
these step sizes the measured ratios are 7-9: the dt^2 term of its error is
still small beside the dt^3 term).  Each difference is held to be many
standard errors from zero, so the ratios are not noise.
"""
import numpy as np
import pytest
import torch

from gpu_util import ensure_built
from paper_0903_3852_gb300 import sde

pytestmark = pytest.mark.gpu

# regular (non-chaotic) regimes with a drift velocity of 0.09-0.18
POINTS = [dict(gamma=3.0, a=4.2, omega=4.9, f=2.0, D=0.1),
          dict(gamma=1.0, a=2.0, omega=3.0, f=0.5, D=0.5)]
PATHS = 1 << 23
PERIODS = 40


def _mean_v(P, flags, x0, v0):
    S = PERIODS * P
    n = x0.numel()
    ens = sde.Ensemble.josephson(POINTS, [PATHS] * len(POINTS), [S] * len(POINTS), 11, steps_per_period=P,
                                 flags=flags)
    xo, vo = torch.empty_like(x0), torch.empty_like(v0)
    wo = torch.empty(n, dtype=torch.int32, device="cuda")
    so = torch.empty(n, dtype=torch.float64, device="cuda")
    ens.run_josephson(0, S, x0, v0, xo, vo, wo, so)
    obs = ens.observables()
    return obs["mean"], obs["se"]


def _ratios(flags, Ps):
    ensure_built()
    rng = np.random.default_rng(0)
    n = PATHS * len(POINTS)
    x0 = torch.from_numpy(rng.random(n).astype(np.float32)).cuda()
    v0 = torch.from_numpy(rng.uniform(-2.0, 2.0, n).astype(np.float32)).cuda()
    (m0, s0), (m1, s1), (m2, s2) = [_mean_v(P, flags, x0, v0) for P in Ps]
    d1, d2 = m0 - m1, m1 - m2
    e1, e2 = np.hypot(s0, s1), np.hypot(s1, s2)
    print("flags %d: differences %s, %s (se %s, %s), ratios %s" % (flags, d1, d2, e1, e2, d1 / d2))
    return d1, d2, e1, e2


def test_srk2_richardson_differences_shrink_faster_than_first_order():
    d1, d2, e1, e2 = _ratios(0, (25, 50, 100))
    assert np.all(np.abs(d2) > 10 * e2) and np.all(np.abs(d1) > 10 * e1)
    assert np.all(d1 / d2 >= 3.0)


def test_euler_richardson_differences_halve():
    d1, d2, e1, e2 = _ratios(sde.SDE_FLAG_EULER, (100, 200, 400))
    assert np.all(np.abs(d2) > 20 * e2)
    r = d1 / d2
    assert np.all((r > 1.6) & (r < 2.8))
