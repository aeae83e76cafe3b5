"""Coarse-grained densities (Fig. 2 and Fig. 4 of the paper) on the GPU.

- Position histograms (bins one potential period wide, Sec. 5): exact integer
  counts of the winding counts, equal to numpy's counts of the same array.
- Phase density: the documented FP32 bin formula replicated in numpy float32 on
  the same phases gives the same counts.
- Sec. 5's claim: single- and double-precision histograms of the Fig. 2
  ensemble agree within statistical error (chi-square two-sample test between
  the GPU's FP32 ensemble and the FP64 oracle's, same noise, chaotic paths).
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

import oracle
from gpu_util import ensure_built, jj_run
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu

FIG2 = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)


def test_position_histogram_exact_counts():
    ensure_built()
    pts = [dict(FIG2, f=0.1 * k) for k in range(4)]
    paths, steps = [3, 0, 700, 129], [2000, 100, 3000, 2500]
    w = inputs.josephson_custom(pts, paths, steps, seed=5)
    ens = sde.Ensemble.josephson(pts, paths, steps, 5, steps_per_period=200)
    *_, wg, xg, sg, obs = jj_run(ens, w["x0"], w["v0"], 0, max(steps))
    w_dev = torch.from_numpy(wg).cuda()
    w_lo, nbins = -3, 7
    counts = ens.position_histogram(w_dev, w_lo, nbins).cpu().numpy()
    off = 0
    for k, n in enumerate(paths):
        ww = wg[off:off + n].astype(np.int64)
        expect = [np.sum(ww < w_lo)] + [np.sum(ww == w_lo + b) for b in range(nbins)] + \
                 [np.sum(ww >= w_lo + nbins)]
        assert counts[k].tolist() == expect
        assert counts[k].sum() == n
        off += n


def test_phase_histogram_matches_fp32_formula():
    ensure_built()
    rng = np.random.default_rng(0)
    nbins = 200
    phi = rng.uniform(0, 2 * np.pi, 100_003).astype(np.float32)
    edges = (np.arange(nbins, dtype=np.float64) * 2 * np.pi / nbins).astype(np.float32)
    phi = np.concatenate([phi, edges, np.nextafter(edges, np.float32(0)), np.float32([0.0, 6.2831850])])
    counts = sde.phase_histogram(torch.from_numpy(phi).cuda(), nbins).cpu().numpy()
    scale = np.float32(nbins / (2 * np.pi))
    b = np.floor((phi * scale).astype(np.float32)).astype(np.int64)
    b = np.clip(b, 0, nbins - 1)
    assert counts.tolist() == np.bincount(b, minlength=nbins).tolist()


def test_fig2_single_and_double_precision_histograms_agree():
    # Fig. 2 setup at reduced size: dt = 0.01 (2 pi / omega), 200 periods
    ensure_built()
    n, P, periods = 2048, 100, 200
    S = P * periods
    w = inputs.josephson_plain(paths=n, steps=S, seed=21)
    ens = sde.Ensemble.josephson([FIG2], [n], [S], 21, steps_per_period=P)
    xg, vg, wg, *_ = jj_run(ens, w["x0"], w["v0"], 0, S)
    xo, vo, _ = oracle.jj_run(w["x0"], w["v0"], oracle.jj_params(**FIG2), P, 0, S, S, 21)
    bg = np.floor(xg).astype(np.int64)
    bo = np.floor(xo).astype(np.int64)
    lo, hi = min(bg.min(), bo.min()), max(bg.max(), bo.max())
    cg = np.bincount(bg - lo, minlength=hi - lo + 1)
    co = np.bincount(bo - lo, minlength=hi - lo + 1)
    keep = (cg + co) >= 10  # pool sparse tail bins
    table = np.array([np.append(cg[keep], cg[~keep].sum()), np.append(co[keep], co[~keep].sum())])
    table = table[:, table.sum(axis=0) > 0]
    chi2, p, dof, _ = stats.chi2_contingency(table)
    agree = np.mean(np.floor(xg) == np.floor(xo))
    print("Fig. 2 histogram: %d bins, chi2 %.1f dof %d p %.3f; same period for %.0f%% of paths" %
          (table.shape[1], chi2, dof, p, 100 * agree))
    assert p > 1e-3
