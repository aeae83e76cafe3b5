"""The grid-wide mean-field form of Eq. 2 (Eq. 3 with each replica spread
over the whole GPU, two launches per step): pathwise parity with the FP64
oracle on ragged sizes, agreement with the one-CTA form, bit-exact resume,
and the paper's Fig. 4 workload at full size (2^24 oscillators, omega_i = 0,
K = 4, T = 1): the first steps against the oracle oscillator by oscillator,
then the stationary state against mean-field theory -- the order parameter
solves r = I1(K r / D) / I0(K r / D) and the phase density is the von Mises
density exp(kappa cos(phi - psi)) / (2 pi I0(kappa)) with kappa = K r / D."""
import math

import numpy as np
import pytest

import oracle
from gpu_util import angle_diff, ensure_built, kur_run
from paper_0903_3852_gb300 import inputs, sde
from test_gpu_kuramoto import _phase_err, _sensitivity

pytestmark = pytest.mark.gpu


def _grid(N, R, K, D, dt, seed, M):
    ensure_built()
    ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_MEANFIELD, N, R, K, D, dt, seed, sample_every=M,
                                schedule=sde.SDE_SCHED_GRID)
    assert ens.tuning()[2] == 0  # grid-wide form
    return ens


@pytest.mark.parametrize("N,R,steps", [(1000, 2, 1000), (100_003, 1, 300), (37, 3, 500)])
def test_grid_meanfield_pathwise(N, R, steps):
    M, seed = 100, 7
    w = inputs.kuramoto_uniform(n_osc=N, replicas=R, seed=3)
    ens = _grid(N, R, 2.0, 0.05, 0.01, seed, M)
    phig, rg, obs = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    worst = 0.0
    for r in range(R):
        phio, ro = oracle.kuramoto_run(w["phi0"][r], w["omega"][r], 0.05, 0.01, 0, steps, seed, r,
                                       Kconst=2.0 / N, meanfield=True, sample_every=M)
        err = _phase_err(phig[r], phio)
        G = _sensitivity(w["phi0"][r], w["omega"][r], 0.05, 0.01, steps, seed, r, 2.0 / N, True, trials=2)
        assert err[G <= 30].max(initial=0.0) <= 1e-5
        assert np.all(err <= 1e-5 + 2e-6 * G)
        worst = max(worst, err[G <= 30].max(initial=0.0))
        assert np.max(np.abs(rg[:, r] - ro)) <= 2e-5
    print("grid meanfield N=%d max phase err (insensitive oscillators) %.2e" % (N, worst))
    assert obs.shape[0] == -(-steps // M) + 1
    assert np.allclose(obs["mean"], rg.mean(axis=1), rtol=0, atol=1e-12)


def test_grid_agrees_with_cta_form_and_resumes():
    N, R, steps = 4096, 3, 400
    w = inputs.kuramoto_uniform(n_osc=N, replicas=R, seed=8)
    a = _grid(N, R, 2.0, 0.05, 0.01, 1, 100)
    b = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_MEANFIELD, N, R, 2.0, 0.05, 0.01, 1, sample_every=100,
                              block_threads=256)
    pa, ra, _ = kur_run(a, w["phi0"], w["omega"], 0, steps)
    pb, rb, _ = kur_run(b, w["phi0"], w["omega"], 0, steps)
    # same Gaussians; only the summation order of S and C differs
    assert np.abs(angle_diff(pa, pb)).max() <= 2e-5
    assert np.abs(ra - rb).max() <= 1e-5
    # split run 0..157, 157..400: the noise counter makes it the same run
    p1, _, _ = kur_run(a, w["phi0"], w["omega"], 0, 157)
    p2, _, _ = kur_run(a, p1.astype(np.float32), w["omega"], 157, steps)
    assert np.abs(angle_diff(p2, pa)).max() <= 2e-6  # phi <-> fixed-point round trip only


def test_grid_zero_steps_and_deterministic():
    N, R = 5000, 2
    w = inputs.kuramoto_uniform(n_osc=N, replicas=R, seed=9)
    ens = _grid(N, R, 2.0, 0.05, 0.01, 3, 10)
    p0, r0, obs = kur_run(ens, w["phi0"], w["omega"], 5, 5)
    assert np.abs(angle_diff(p0, w["phi0"])).max() <= 1e-6
    assert r0.shape[0] == 1 and obs.shape[0] == 1
    for r in range(R):
        z = np.exp(1j * w["phi0"][r].astype(np.float64))
        assert abs(r0[0, r] - abs(z.mean())) <= 1e-6
    p1, r1, _ = kur_run(ens, w["phi0"], w["omega"], 0, 123)
    p2, r2, _ = kur_run(ens, w["phi0"], w["omega"], 0, 123)
    assert np.array_equal(p1, p2) and np.array_equal(r1, r2)  # fixed-order reductions


def test_fig4_first_steps_full_size():
    w = inputs.kuramoto_fig4()
    N, steps = w["n_osc"], 3
    ens = _grid(N, 1, w["K"], w["D"], w["dt"], w["seed"], 1)
    phig, rg, _ = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    phio, ro = oracle.kuramoto_run(w["phi0"][0], w["omega"][0], w["D"], w["dt"], 0, steps, w["seed"], 0,
                                   Kconst=w["K"] / N, meanfield=True, sample_every=1)
    err = _phase_err(phig[0], phio)
    print("fig4 %d oscillators, %d steps: max phase err %.2e" % (N, steps, err.max()))
    assert err.max() <= 1e-5
    assert np.max(np.abs(rg[:, 0] - ro)) <= 1e-6


def _r_star(k_over_d):
    from scipy.optimize import brentq
    from scipy.special import i0e, i1e
    return brentq(lambda r: r - i1e(k_over_d * r) / i0e(k_over_d * r), 1e-3, 1 - 1e-9)


def test_fig4_stationary_state_full_size():
    pytest.importorskip("scipy")
    from scipy.special import i0e
    w = inputs.kuramoto_fig4()
    N, S, M = w["n_osc"], w["steps"], w["sample_every"]
    ens = _grid(N, 1, w["K"], w["D"], w["dt"], w["seed"], M)
    phig, rg, obs = kur_run(ens, w["phi0"], w["omega"], 0, S)
    r_inf = _r_star(w["K"] / w["D"])
    late = rg[-5:, 0]
    print("fig4 r(t) late %s, theory %.5f" % (np.array2string(late, precision=5), r_inf))
    assert rg[0, 0] < 0.01  # uniform start
    assert np.all(np.abs(late - r_inf) <= 3e-3)
    # phase density against the von Mises law around the mean phase
    import torch
    nb = 128
    counts = sde.phase_histogram(torch.from_numpy(phig[0].astype(np.float32)).cuda(), nb).cpu().numpy()
    assert counts.sum() == N
    psi = math.atan2(np.sin(phig[0]).mean(), np.cos(phig[0]).mean())
    kappa = w["K"] * r_inf / w["D"]
    edges = np.linspace(0.0, 2 * np.pi, nb + 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    p = np.exp(kappa * (np.cos(mid - psi) - 1.0)) / (2 * np.pi * i0e(kappa)) * (2 * np.pi / nb)
    tv = 0.5 * np.abs(counts / N - p / p.sum()).sum()
    print("fig4 phase density total variation vs von Mises %.4f" % tv)
    assert tv <= 0.01
