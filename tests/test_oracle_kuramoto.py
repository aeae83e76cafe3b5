"""Pins of the oracle's Eq. 2 integrator and coupling sums (CPU only).

- Eq. 3: the direct pairwise sum equals the mean-field form for uniform K.
- General K: for a rank-one matrix K_ij = alpha_i beta_j the sum has the
  closed form alpha_i (cos phi_i sum_j beta_j sin phi_j - sin phi_i sum_j
  beta_j cos phi_j); a transposed K (K_ji) fails it.
- Sign of the coupling (Eq. 2 uses sin(x_j - x_i)): attractive coupling
  synchronises identical oscillators (r -> 1).
- Two oscillators, D = 0: the phase difference obeys Adler's equation
  d' = dw - K sin d, whose fixed point is arcsin(dw / K); the trajectory
  converges to a DOP853 solution with order 2.
- Free diffusion (K = 0, omega = 0): phi(t) - phi(0) = sqrt(2D) W(t), so
  Var = 2 D t (the <x^2> = 2Dt check); with omega != 0 the drift is exact.
- Order parameter closed forms.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

import oracle


def test_meanfield_identity_eq3():
    rng = np.random.default_rng(1)
    for N in (1, 7, 512, 4096):
        phi = rng.uniform(0, 2 * np.pi, N) + rng.integers(-3, 3, N) * 2 * np.pi
        d = oracle.coupling_direct(phi, Kconst=1.7)
        m = oracle.coupling_meanfield(phi, 1.7)
        scale = 1.7 * N
        assert np.max(np.abs(d - m)) <= 1e-12 * scale


def test_general_coupling_rank_one_closed_form():
    rng = np.random.default_rng(2)
    N = 300
    phi = rng.uniform(0, 2 * np.pi, N)
    alpha, beta = rng.uniform(0.5, 1.5, N), rng.uniform(-1, 1, N)
    K = np.outer(alpha, beta)
    got = oracle.coupling_direct(phi, Kmat=K)
    expect = alpha * (np.cos(phi) * np.dot(beta, np.sin(phi)) - np.sin(phi) * np.dot(beta, np.cos(phi)))
    assert np.max(np.abs(got - expect)) < 1e-12 * N
    transposed = oracle.coupling_direct(phi, Kmat=K.T)
    assert np.max(np.abs(transposed - expect)) > 1e-2


def test_uniform_matrix_equals_constant():
    rng = np.random.default_rng(3)
    N = 64
    phi = rng.uniform(0, 2 * np.pi, N)
    a = oracle.coupling_direct(phi, Kmat=np.full((N, N), 0.25))
    b = oracle.coupling_direct(phi, Kconst=0.25)
    assert np.array_equal(a, b)


def test_order_parameter_closed_forms():
    assert abs(oracle.order_parameter(np.full(10, 1.234)) - 1.0) < 1e-15
    N = 17
    assert oracle.order_parameter(2 * np.pi * np.arange(N) / N) < 1e-15
    for d in (0.1, 1.0, 2.5):
        assert abs(oracle.order_parameter([0.3, 0.3 + d]) - abs(math.cos(d / 2))) < 1e-15


def test_attractive_coupling_synchronises():
    rng = np.random.default_rng(4)
    N, K = 64, 2.0
    phi0 = rng.uniform(0, 2 * np.pi, N)
    omega = np.zeros(N)
    for meanfield in (False, True):
        phi, r = oracle.kuramoto_run(phi0, omega, D=0.0, dt=0.01, n_begin=0, n_end=2000,
                                     seed=0, replica=0, Kconst=K / N, meanfield=meanfield,
                                     sample_every=100)
        assert r[0] == oracle.order_parameter(phi0)
        assert r[-1] > 0.999
        assert np.all(np.diff(r) > -1e-12)  # r never decreases for identical oscillators


def _adler_two(omega, K, d0, t_end):
    # phase difference d = phi_2 - phi_1 of two oscillators with K_ij = K / 2
    sol = solve_ivp(lambda t, y: [(omega[1] - omega[0]) - K * math.sin(y[0])], (0, t_end),
                    [d0], method="DOP853", rtol=1e-13, atol=1e-13)
    return sol.y[0, -1]


def test_two_oscillators_adler_equation():
    omega = np.array([-0.3, 0.5])
    K = 2.0
    phi0 = np.array([0.2, 2.9])
    # fixed point of d' = dw - K sin d
    phi, _ = oracle.kuramoto_run(phi0, omega, 0.0, 0.01, 0, 5000, 0, 0, Kconst=K / 2)
    d_star = math.asin((omega[1] - omega[0]) / K)
    assert abs((phi[1] - phi[0]) - d_star) < 1e-9
    # locked pair moves with the mean frequency
    # convergence of the difference to the exact ODE, order 2
    t_end = 2.0
    ref = _adler_two(omega, K, phi0[1] - phi0[0], t_end)
    errs = []
    for dt in (0.02, 0.01, 0.005, 0.0025):
        phi, _ = oracle.kuramoto_run(phi0, omega, 0.0, dt, 0, int(round(t_end / dt)), 0, 0,
                                     Kconst=K / 2)
        errs.append(abs((phi[1] - phi[0]) - ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - 2.0) < 0.1 for s in slopes), (errs, slopes)


def test_free_diffusion_variance_is_2Dt():
    N, D, dt, steps = 20_000, 0.05, 0.01, 200
    phi0 = np.zeros(N)
    phi, _ = oracle.kuramoto_run(phi0, np.zeros(N), D, dt, 0, steps, seed=11, replica=3,
                                 Kconst=0.0, meanfield=True)
    t = steps * dt
    var = np.mean(phi ** 2)
    se = 2 * D * t * math.sqrt(2.0 / N)
    assert abs(var - 2 * D * t) < 4 * se
    assert abs(phi.mean()) < 4 * math.sqrt(2 * D * t / N)


def test_free_rotation_is_exact_and_noise_stream_layout():
    N, D, dt, steps = 8, 0.0, 0.01, 37
    omega = np.linspace(-1, 1, N)
    phi0 = np.linspace(0, 1, N)
    phi, _ = oracle.kuramoto_run(phi0, omega, D, dt, 0, steps, 0, 0, Kconst=0.0)
    assert np.max(np.abs(phi - (phi0 + omega * steps * dt))) < 1e-13
    # one step with noise: phi1 - phi0 = omega dt + sqrt(2 D dt) psi_{i, r, n}
    D = 0.3
    phi, _ = oracle.kuramoto_run(phi0, omega, D, dt, 5, 6, seed=42, replica=9, Kconst=0.0)
    psi = np.array([oracle.gaussian(42, oracle.TAG_KURAMOTO, i, 9, 5) for i in range(N)])
    assert np.max(np.abs(phi - phi0 - omega * dt - math.sqrt(2 * D * dt) * psi)) < 1e-14


def test_run_resumes_bit_exactly_and_samples():
    rng = np.random.default_rng(5)
    N = 32
    phi0, omega = rng.uniform(0, 2 * np.pi, N), rng.normal(size=N)
    a, ra = oracle.kuramoto_run(phi0, omega, 0.05, 0.01, 0, 300, 1, 2, Kconst=2.0 / N,
                                sample_every=100)
    b, _ = oracle.kuramoto_run(phi0, omega, 0.05, 0.01, 0, 100, 1, 2, Kconst=2.0 / N)
    b, rb = oracle.kuramoto_run(b, omega, 0.05, 0.01, 100, 300, 1, 2, Kconst=2.0 / N,
                                sample_every=100)
    assert np.array_equal(a, b)
    assert ra.shape == (4,) and np.array_equal(ra[1:], rb)
    assert ra[-1] == oracle.order_parameter(a)
