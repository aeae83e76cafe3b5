"""Pins of the oracle's Euler-Maruyama scheme (the first-order scheme of the
paper's PROG2, Sec. 4.2), CPU only.

- D = 0: the step reduces to the explicit Euler method; it must converge to a
  high-accuracy ODE solution (scipy DOP853) with global order 1, for Eq. 1
  and for the two-oscillator Kuramoto system (Adler's equation).
- Weak order 1: for a linear force the step is an affine map plus a Gaussian,
  so mean and covariance propagate exactly; they approach the exact moments
  of the continuous process (Van Loan) with error ratio ~2 per halving of dt,
  and the stationary covariance misses equipartition by O(dt).
- Constant drift (K = 0): Euler and SRK2 coincide exactly, and one step is
  omega dt + sqrt(2 D dt) psi with psi the noise stream's Gaussian.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

import oracle
from test_oracle_josephson import CFG1, _exact_ode, _vanloan_moments


def test_euler_deterministic_limit_converges_with_order_one():
    p = oracle.jj_params(**{**CFG1, "D": 0.0})
    T = 2 * math.pi / p.omega
    ref = _exact_ode(p, 0.3, 0.5, T)
    errs = []
    for P in (3200, 6400, 12800, 25600):
        x, v, _ = oracle.jj_run([0.3], [0.5], p, P, 0, P, P, seed=0, scheme=oracle.SCHEME_EULER)
        errs.append(math.hypot(x[0] - ref[0], v[0] - ref[1]))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - 1.0) < 0.1 for s in slopes), (errs, slopes)


def _euler_affine_map(dt, gamma, kappa, f, D):
    """Read the Euler step off the oracle: y' = A y + b + c psi."""
    st = lambda x, v, z: np.array(oracle.linear_euler_step(x, v, dt, gamma, kappa, f, D, z))
    y0 = st(0.0, 0.0, 0.0)
    A = np.stack([st(1.0, 0.0, 0.0) - y0, st(0.0, 1.0, 0.0) - y0], axis=1)
    return A, y0, st(0.0, 0.0, 1.0) - y0


def test_euler_step_is_first_order_taylor_with_noise_on_v():
    gamma, kappa, f, D, dt = 0.9, 4.0, 0.1, 0.05, 0.01
    A, b, c = _euler_affine_map(dt, gamma, kappa, f, D)
    # x' = x + dt v; v' = v + dt(-gamma v - kappa x + f) + sqrt(2 gamma D dt) psi
    assert np.allclose(A, np.eye(2) + dt * np.array([[0.0, 1.0], [-kappa, -gamma]]), rtol=0, atol=1e-15)
    assert np.allclose(b, [0.0, dt * f], rtol=0, atol=1e-16)
    assert abs(c[0]) == 0.0 and abs(c[1] - math.sqrt(2 * gamma * D * dt)) < 1e-15


def test_euler_weak_order_one_linear_model():
    gamma, kappa, f, D = 0.9, 4.0, 0.1, 0.05
    M = np.array([[0.0, 1.0], [-kappa, -gamma]])
    G = np.array([0.0, math.sqrt(2 * gamma * D)])
    m0 = np.array([1.0, 0.0])
    T = 2.0
    m_ex, c_ex = _vanloan_moments(M, np.array([0.0, f]), G, m0, T)
    errs = []
    for dt in (0.004, 0.002, 0.001, 0.0005):
        A, bd, c = _euler_affine_map(dt, gamma, kappa, f, D)
        m, C = m0.copy(), np.zeros((2, 2))
        for _ in range(int(round(T / dt))):
            m = A @ m + bd
            C = A @ C @ A.T + np.outer(c, c)
        errs.append(np.abs(m - m_ex).max() + np.abs(C - c_ex).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in ratios), (errs, ratios)


def test_euler_stationary_covariance_misses_equipartition_by_order_dt():
    gamma, kappa, f, D = 0.9, 4.0, 0.1, 0.05
    bias = []
    for dt in (0.002, 0.001):
        A, bd, c = _euler_affine_map(dt, gamma, kappa, f, D)
        m, C = np.zeros(2), np.zeros((2, 2))
        for _ in range(int(40.0 / dt)):
            m = A @ m + bd
            C = A @ C @ A.T + np.outer(c, c)
        assert abs(m[0] - f / kappa) < 1e-9 and abs(m[1]) < 1e-9  # the mean is exact
        bias.append(abs(C[1, 1] - D) / D)
    assert 1.8 < bias[0] / bias[1] < 2.2 and bias[0] < 0.01


def _adler_two(omega, K, d0, t_end):
    sol = solve_ivp(lambda t, y: [(omega[1] - omega[0]) - K * math.sin(y[0])], (0, t_end), [d0],
                    method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[0, -1]


def test_euler_kuramoto_two_oscillators_order_one():
    omega = np.array([-0.3, 0.5])
    K = 2.0
    phi0 = np.array([0.2, 2.9])
    t_end = 2.0
    ref = _adler_two(omega, K, phi0[1] - phi0[0], t_end)
    errs = []
    for dt in (0.004, 0.002, 0.001, 0.0005):
        phi, _ = oracle.kuramoto_run(phi0, omega, 0.0, dt, 0, int(round(t_end / dt)), 0, 0, Kconst=K / 2,
                                     scheme=oracle.SCHEME_EULER)
        errs.append(abs((phi[1] - phi[0]) - ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - 1.0) < 0.1 for s in slopes), (errs, slopes)
    # the locked fixed point is the same as the continuous one
    phi, _ = oracle.kuramoto_run(phi0, omega, 0.0, 0.01, 0, 5000, 0, 0, Kconst=K / 2, scheme=oracle.SCHEME_EULER)
    assert abs((phi[1] - phi[0]) - math.asin((omega[1] - omega[0]) / K)) < 1e-9


def test_euler_equals_srk2_for_constant_drift_and_uses_the_noise_stream():
    N, D, dt = 16, 0.3, 0.01
    omega = np.linspace(-1, 1, N)
    phi0 = np.linspace(0, 1, N)
    a, _ = oracle.kuramoto_run(phi0, omega, D, dt, 3, 40, 42, 9, Kconst=0.0, scheme=oracle.SCHEME_EULER)
    b, _ = oracle.kuramoto_run(phi0, omega, D, dt, 3, 40, 42, 9, Kconst=0.0)
    assert np.array_equal(a, b)
    phi, _ = oracle.kuramoto_run(phi0, omega, D, dt, 5, 6, 42, 9, Kconst=0.0, scheme=oracle.SCHEME_EULER)
    psi = np.array([oracle.gaussian(42, oracle.TAG_KURAMOTO, i, 9, 5) for i in range(N)])
    assert np.max(np.abs(phi - phi0 - omega * dt - math.sqrt(2 * D * dt) * psi)) < 1e-14


def test_euler_josephson_resumes_bit_exactly_and_noise_slope():
    p = oracle.jj_params(**CFG1)
    x0, v0 = np.linspace(0, 1, 7), np.linspace(-1, 1, 7)
    a = oracle.jj_run(x0, v0, p, 200, 0, 300, 300, 3, scheme=oracle.SCHEME_EULER)
    b1 = oracle.jj_run(x0, v0, p, 200, 0, 123, 300, 3, scheme=oracle.SCHEME_EULER)
    b = oracle.jj_run(b1[0], b1[1], p, 200, 123, 300, 300, 3, vsum=b1[2], scheme=oracle.SCHEME_EULER)
    for u, w in zip(a, b):
        assert np.array_equal(u, w)
    dt = 2 * math.pi / (p.omega * 200)
    s = math.sqrt(2 * p.gamma * p.D * dt)
    x_a, v_a = oracle.jj_euler_step(0.3, 0.5, 7, dt, p, 0.0)
    x_b, v_b = oracle.jj_euler_step(0.3, 0.5, 7, dt, p, 1.0)
    assert x_a == x_b and abs((v_b - v_a) - s) < 1e-15
