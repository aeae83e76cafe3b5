"""The seeded input recipes: sizes, ranges and orderings of the synthetic
workloads (the readings of the workload definitions), and determinism."""
import math

import numpy as np

from paper_0903_3852_gb300 import inputs


def test_sweep_grid_is_the_first_512_of_171_f_by_3_D_pairs_D_major():
    pts = inputs.sweep_grid()
    assert len(pts) == 512
    f = np.linspace(0.0, 0.5, 171)
    for i, p in enumerate(pts):
        d, k = divmod(i, 171)
        assert p["D"] == (1e-4, 1e-3, 1e-2)[d] and p["f"] == f[k]
        assert (p["gamma"], p["a"], p["omega"]) == (0.9, 4.2, 4.9)
    assert pts[-1]["D"] == 1e-2 and pts[-1]["f"] == f[169]  # the 513th pair is the one left out


def test_sweep_sizes_are_log_uniform_in_their_ranges_and_reproducible():
    w, w2 = inputs.josephson_sweep(), inputs.josephson_sweep()
    assert np.array_equal(w["paths"], w2["paths"]) and np.array_equal(w["x0"], w2["x0"])
    p, s = w["paths"], w["steps"]
    assert p.min() >= 256 and p.max() <= 8192 and s.min() >= 10_000 and s.max() <= 100_000
    # log-uniform: the logs are spread evenly over the range (mean near the middle)
    for a, (lo, hi) in ((p, (256, 8192)), (s, (10_000, 100_000))):
        u = (np.log(a) - math.log(lo)) / (math.log(hi) - math.log(lo))
        assert abs(u.mean() - 0.5) < 0.05 and 0.05 < u.std() < 0.4
    assert int(p.sum()) == 1_127_520 and float((p * s).sum()) == 46_746_724_836.0
    assert w["x0"].size == p.sum() and (w["x0"] >= 0).all() and (w["x0"] < 1).all()
    assert (np.abs(w["v0"]) <= 2).all()


def test_fig2_and_fig4_ensembles():
    w = inputs.josephson_fig2()
    assert int(w["paths"][0]) == 2 ** 19 and int(w["steps"][0]) == 200_000 and w["steps_per_period"] == 100
    k = inputs.kuramoto_fig4()
    assert k["n_osc"] == 2 ** 24 and k["replicas"] == 1 and not k["omega"].any()
    # drawn in [0, 2 pi) in FP64; the FP32 cast can round up to 2 pi itself (= 0 as an angle)
    assert (k["phi0"] >= 0).all() and (k["phi0"] <= np.float32(2 * math.pi)).all()


def test_kuramoto_uniform_frequencies_are_independent_per_replica():
    k = inputs.kuramoto_uniform(n_osc=256, replicas=8, seed=3)
    om = k["omega"]
    assert om.shape == (8, 256)
    assert abs(om.mean()) < 0.1 and abs(om.std() - 1.0) < 0.1
    assert not np.array_equal(om[0], om[1])
