"""Euler-Maruyama on the GPU (SDE_FLAG_EULER, the first-order scheme of
PROG2, Sec. 4.2) against the oracle's Euler-Maruyama with identical
Gaussians: Josephson on every schedule, and the pairwise Kuramoto model as
PROG2's two kernels per step (UpdateRHS, AdvanceSystem)."""
import numpy as np
import pytest

import oracle
from gpu_util import angle_diff, ensure_built, jj_run, kur_run, mixed_rel
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu

FIG2 = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)
DAMPED = dict(gamma=2.5, a=0.8, omega=1.3, f=0.35, D=2e-3)
EM = oracle.SCHEME_EULER


@pytest.mark.parametrize("schedule", [sde.SDE_SCHED_PERSISTENT, sde.SDE_SCHED_PLAIN])
def test_josephson_euler_matches_oracle(schedule):
    ensure_built()
    pts = [DAMPED, dict(DAMPED, f=0.0, a=1.7), dict(FIG2)]
    paths, steps = [300, 77, 129], [600, 401, 100]
    w = inputs.josephson_custom(pts, paths, steps, seed=3)
    ens = sde.Ensemble.josephson(pts, paths, steps, 3, steps_per_period=200, schedule=schedule,
                                 flags=sde.SDE_FLAG_EULER)
    xg, vg, wg, xf, sg, obs = jj_run(ens, w["x0"], w["v0"], 0, max(steps))
    off = 0
    for k, (pt, n, S) in enumerate(zip(pts, paths, steps)):
        sl = slice(off, off + n)
        xo, vo, so = oracle.jj_run(w["x0"][sl], w["v0"][sl], oracle.jj_params(**pt), 200, 0, S, S, 3, point=k,
                                   scheme=EM)
        ex, ev = mixed_rel(xg[sl], xo).max(), mixed_rel(vg[sl], vo).max()
        W = S // 2
        ea = np.abs(sg[sl] / W - so / W).max()
        print("euler point %d: x %.2e v %.2e <v>_path %.2e" % (k, ex, ev, ea))
        assert ex <= 1e-5 and ev <= 1e-5 and ea <= 1e-5
        assert abs(obs["mean"][k] - (so / W).mean()) <= 1e-5
        off += n


def test_josephson_euler_differs_from_srk2_by_order_dt():
    # one step from the same state: the two schemes differ by O(dt^2) in x
    ensure_built()
    n = 256
    w = inputs.josephson_plain(paths=n, steps=1)
    a = sde.Ensemble.josephson([FIG2], [n], [1], 0, steps_per_period=200, flags=sde.SDE_FLAG_EULER)
    b = sde.Ensemble.josephson([FIG2], [n], [1], 0, steps_per_period=200)
    xa, va, *_ = jj_run(a, w["x0"], w["v0"], 0, 1)
    xb, vb, *_ = jj_run(b, w["x0"], w["v0"], 0, 1)
    dt = 2 * np.pi / (4.9 * 200)
    dx = np.abs(xa - xb).max()
    assert 1e-3 * dt * dt < dx < 30 * dt * dt


@pytest.mark.parametrize("N,R", [(300, 2), (1024, 1)])
def test_kuramoto_pairwise_euler_prog2_split(N, R):
    ensure_built()
    steps, M, seed = 203, 50, 5
    w = inputs.kuramoto_uniform(n_osc=N, replicas=R, seed=6)
    ens = sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_PAIRWISE, N, R, 2.0, 0.05, 0.01, seed, sample_every=M,
                                flags=sde.SDE_FLAG_EULER)
    phig, rg, obs = kur_run(ens, w["phi0"], w["omega"], 0, steps)
    for r in range(R):
        phio, ro = oracle.kuramoto_run(w["phi0"][r], w["omega"][r], 0.05, 0.01, 0, steps, seed, r,
                                       Kconst=2.0 / N, sample_every=M, scheme=EM)
        err = np.abs(angle_diff(phig[r], phio)) / np.maximum(1.0, np.mod(phio, 2 * np.pi))
        print("pairwise euler N=%d max phase err %.2e" % (N, err.max()))
        assert err.max() <= 1e-5
        assert np.max(np.abs(rg[:, r] - ro)) <= 2e-5


def test_euler_unsupported_models_are_rejected():
    ensure_built()
    for model in (sde.SDE_KURAMOTO_MEANFIELD, sde.SDE_KURAMOTO_GENERAL):
        with pytest.raises(sde.SDEError) as e:
            sde.Ensemble.kuramoto(model, 64, 1, 2.0, 0.05, 0.01, 0, flags=sde.SDE_FLAG_EULER)
        assert e.value.status == sde.SDE_ERR_UNSUPPORTED
