"""Pins of the oracle's Eq. 1 integrator (CPU only).

- D = 0: the SRK2 step of Alg. 2 reduces to Heun's method; it must converge to
  a high-accuracy ODE solution (scipy DOP853) with global order 2.
- Noise placement: for additive noise the step is affine in psi with slopes
  that follow from Alg. 2 applied to (x, v) with noise sqrt(2 gamma D) on v.
- Weak order 2 and the noise amplitude: for a linear force the step is an
  affine map plus a Gaussian, so mean and covariance propagate exactly; they
  must approach the exact moments of the continuous process (Van Loan's
  matrix exponential, itself pinned to the Uhlenbeck-Ornstein closed form)
  with error ratio ~4 per halving of dt, and the stationary covariance must be
  the equipartition value diag(D/kappa, D).
- The averaging window of <v> (time average over the last half of the run).
"""
import math

import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.linalg import expm

import oracle

CFG1 = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=0.001)


def _exact_ode(p, x0, v0, t_end):
    sol = solve_ivp(lambda t, y: oracle.jj_rhs(t, y, p), (0.0, t_end), [x0, v0],
                    method="DOP853", rtol=1e-13, atol=1e-13)
    assert sol.success
    return sol.y[:, -1]


def test_deterministic_limit_converges_with_order_two():
    p = oracle.jj_params(**{**CFG1, "D": 0.0})
    # Two drive periods: beyond that, the deterministic dynamics at these
    # parameters amplify step errors strongly (the sensitivity noted in
    # Sec. 5), and the asymptotic regime needs a far finer dt.
    periods = 2
    T = 2 * math.pi / p.omega
    ref = _exact_ode(p, 0.3, 0.5, periods * T)
    errs = []
    for P in (200, 400, 800, 1600, 3200):
        x, v, _ = oracle.jj_run([0.3], [0.5], p, P, 0, periods * P, periods * P, seed=0)
        errs.append(math.hypot(x[0] - ref[0], v[0] - ref[1]))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - 2.0) < 0.1 for s in slopes), (errs, slopes)
    assert errs[0] < 1e-2


def test_drive_phase_and_bias_enter_with_the_right_sign():
    # Without potential-dominated motion the drive and bias shift v linearly;
    # compare the one-step change with the exact ODE over one step at tiny dt.
    p = oracle.jj_params(**{**CFG1, "D": 0.0})
    for x0, v0 in ((0.1, 0.0), (0.7, -1.3), (0.25, 2.0)):
        dt = 1e-5
        ref = _exact_ode(p, x0, v0, dt)
        x1, v1 = oracle.jj_step(x0, v0, 0, dt, p, 0.0)
        assert abs(x1 - ref[0]) < 1e-11 and abs(v1 - ref[1]) < 1e-11


def test_noise_enters_affinely_with_closed_form_slopes():
    p = oracle.jj_params(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=0.37)
    dt = 0.0123
    s = math.sqrt(2 * p.gamma * p.D * dt)
    for n, (x0, v0) in enumerate(((0.3, 0.5), (0.9, -2.0), (-3.2, 1.1))):
        x_a, v_a = oracle.jj_step(x0, v0, n, dt, p, 0.0)
        x_b, v_b = oracle.jj_step(x0, v0, n, dt, p, 1.0)
        x_c, v_c = oracle.jj_step(x0, v0, n, dt, p, -2.5)
        assert abs((x_b - x_a) - 0.5 * dt * s) < 1e-14
        assert abs((v_b - v_a) - s * (1.0 - 0.5 * p.gamma * dt)) < 1e-13
        # affine: the psi = -2.5 point lies on the same line
        assert abs((v_c - v_a) + 2.5 * (v_b - v_a)) < 1e-13
        assert abs((x_c - x_a) + 2.5 * (x_b - x_a)) < 1e-15


def _vanloan_moments(M, b, G, m0, t):
    n = M.shape[0]
    Maug = np.zeros((n + 1, n + 1))
    Maug[:n, :n] = M
    Maug[:n, n] = b
    mean = (expm(Maug * t) @ np.append(m0, 1.0))[:n]
    C = np.zeros((2 * n, 2 * n))
    C[:n, :n] = -M
    C[:n, n:] = np.outer(G, G)
    C[n:, n:] = M.T
    E = expm(C * t)
    Phi = E[n:, n:].T
    cov = Phi @ E[:n, n:]
    return mean, 0.5 * (cov + cov.T)


def test_vanloan_matches_uhlenbeck_ornstein_closed_form():
    # Free particle with friction (kappa = 0), x0 = v0 = 0:
    # Var x(t) = (2D/gamma) [t - 2(1 - e^{-gamma t})/gamma + (1 - e^{-2 gamma t})/(2 gamma)]
    # Var v(t) = D (1 - e^{-2 gamma t})
    gamma, D = 0.9, 0.05
    M = np.array([[0.0, 1.0], [0.0, -gamma]])
    G = np.array([0.0, math.sqrt(2 * gamma * D)])
    for t in (0.1, 1.0, 7.5):
        _, cov = _vanloan_moments(M, np.zeros(2), G, np.zeros(2), t)
        varx = (2 * D / gamma) * (t - 2 * (1 - math.exp(-gamma * t)) / gamma
                                  + (1 - math.exp(-2 * gamma * t)) / (2 * gamma))
        varv = D * (1 - math.exp(-2 * gamma * t))
        assert abs(cov[0, 0] - varx) < 1e-12 * max(1, varx)
        assert abs(cov[1, 1] - varv) < 1e-13


def _scheme_affine_map(dt, gamma, kappa, f, D):
    """Read the SRK2 step off the oracle: y' = A y + b + c psi."""
    y0 = np.array(oracle.linear_step(0.0, 0.0, dt, gamma, kappa, f, D, 0.0))
    A = np.zeros((2, 2))
    A[:, 0] = np.array(oracle.linear_step(1.0, 0.0, dt, gamma, kappa, f, D, 0.0)) - y0
    A[:, 1] = np.array(oracle.linear_step(0.0, 1.0, dt, gamma, kappa, f, D, 0.0)) - y0
    c = np.array(oracle.linear_step(0.0, 0.0, dt, gamma, kappa, f, D, 1.0)) - y0
    return A, y0, c


def test_weak_order_two_linear_model():
    gamma, kappa, f, D = 0.9, 4.0, 0.1, 0.05
    M = np.array([[0.0, 1.0], [-kappa, -gamma]])
    b = np.array([0.0, f])
    G = np.array([0.0, math.sqrt(2 * gamma * D)])
    m0 = np.array([1.0, 0.0])
    T = 2.0
    m_ex, c_ex = _vanloan_moments(M, b, G, m0, T)
    errs = []
    for dt in (0.02, 0.01, 0.005, 0.0025):
        A, bd, c = _scheme_affine_map(dt, gamma, kappa, f, D)
        m, C = m0.copy(), np.zeros((2, 2))
        for _ in range(int(round(T / dt))):
            m = A @ m + bd
            C = A @ C @ A.T + np.outer(c, c)
        errs.append(np.abs(m - m_ex).max() + np.abs(C - c_ex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.6 < r < 4.4 for r in ratios), (errs, ratios)


def test_stationary_covariance_is_equipartition():
    gamma, kappa, f, D = 0.9, 4.0, 0.1, 0.05
    dt = 0.001
    A, bd, c = _scheme_affine_map(dt, gamma, kappa, f, D)
    m, C = np.zeros(2), np.zeros((2, 2))
    for _ in range(40_000):
        m = A @ m + bd
        C = A @ C @ A.T + np.outer(c, c)
    assert abs(m[0] - f / kappa) < 1e-9 and abs(m[1]) < 1e-9
    assert abs(C[0, 0] - D / kappa) < 1e-5 * D and abs(C[1, 1] - D) < 1e-5 * D
    assert abs(C[0, 1]) < 1e-5 * D


def test_one_step_ensemble_uses_unit_gaussian_noise():
    # From one state, one step of many paths: v1 is affine in psi, so
    # Var v1 = (s (1 - gamma dt / 2))^2 exactly for unit-variance noise.
    p = oracle.jj_params(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=0.5)
    P = 200
    dt = 2 * math.pi / (p.omega * P)
    n_paths = 40_000
    x, v, _ = oracle.jj_run(np.full(n_paths, 0.2), np.full(n_paths, 0.3), p, P, 6, 7, 100,
                            seed=99, point=3)
    s = math.sqrt(2 * p.gamma * p.D * dt) * (1 - 0.5 * p.gamma * dt)
    x0, v0 = oracle.jj_step(0.2, 0.3, 6, dt, p, 0.0)
    z = (v - v0) / s
    assert abs(z.mean()) < 4 / math.sqrt(n_paths)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n_paths)
    # path j of point k uses stream (c1 = j, c2 = k)
    assert abs(z[17] - oracle.gaussian(99, oracle.TAG_JOSEPHSON, 17, 3, 6)) < 1e-9


def test_window_average_matches_displacement():
    # D = 0: sum over the window of v(t_n) dt equals x(t_S) - x(t_S - W dt)
    # + dt/2 (v_S - v_{S-W}) up to O(dt^2) (trapezoid rule), with the exact
    # trajectory from DOP853.
    p = oracle.jj_params(**{**CFG1, "D": 0.0})
    P, S = 3200, 3200  # one drive period at a fine step: SRK2 tracks the ODE
    W = S // 2
    dt = 2 * math.pi / (p.omega * P)
    x, v, vs = oracle.jj_run([0.3], [0.5], p, P, 0, S, S, seed=0)
    ya = _exact_ode(p, 0.3, 0.5, (S - W) * dt)
    yb = _exact_ode(p, 0.3, 0.5, S * dt)
    expect = (yb[0] - ya[0]) + 0.5 * dt * (yb[1] - ya[1])
    tol = 1e-5
    assert abs(vs[0] * dt - expect) < tol
    # a window shifted by one step would be off by dt * (v_S - v_{S-W}):
    assert dt * abs(yb[1] - ya[1]) > 10 * tol


def test_run_resumes_bit_exactly():
    p = oracle.jj_params(**CFG1)
    rng = np.random.default_rng(0)
    x0, v0 = rng.random(8), rng.uniform(-2, 2, 8)
    S = 1000
    xa, va, sa = oracle.jj_run(x0, v0, p, 200, 0, S, S, seed=5, point=2, path0=10)
    xb, vb, sb = oracle.jj_run(x0, v0, p, 200, 0, 437, S, seed=5, point=2, path0=10)
    xb, vb, sb = oracle.jj_run(xb, vb, p, 200, 437, S, S, seed=5, point=2, path0=10, vsum=sb)
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(sa, sb)
