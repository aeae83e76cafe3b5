"""The FP64 GPU path of Eq. 1 (sde_josephson_run_fp64): Alg. 2 in double
precision with the FP32 path's noise stream.

- Against the FP64 oracle (same algorithm, same Gaussians up to libm/CUDA
  rounding): 1e-11 on a damped point where differences do not grow; at the
  chaotic Fig. 2 parameters 1e-12 over one drive period, and over ten
  periods each path within 100 times the oracle's own divergence under
  FP64-rounding-sized jitter (rounding differences grow by the Lyapunov
  factor, Sec. 5).
- Splitting a run at any step reproduces it bit for bit.
- Sec. 5's comparison on the GPU itself: the FP32 ensemble and the FP64
  ensemble of the Fig. 2 setup (2^16 paths, 200 periods) give the same
  coarse-grained histogram (chi-square two-sample) and <v> within 3 SE.
"""
import numpy as np
import pytest
import torch
from scipy import stats

import oracle
from gpu_util import ensure_built, jj_run
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu

FIG2 = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)
DAMPED = dict(gamma=2.5, a=0.8, omega=1.3, f=0.35, D=2e-3)


def _run64(point, P, S, seed, x0, v0, n_begin=0, n_end=None, vsum=None, point_index=0, state=None):
    n_end = S if n_end is None else n_end
    if state is None:
        x = torch.from_numpy(np.asarray(x0, np.float64)).cuda()
        v = torch.from_numpy(np.asarray(v0, np.float64)).cuda()
        vs = torch.zeros_like(x) if vsum is None else torch.from_numpy(np.asarray(vsum, np.float64)).cuda()
    else:
        x, v, vs = state
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    sde.josephson_run_fp64(point, P, S, seed, n_begin, n_end, x, v, x, v, vsum_in=vs, vsum_out=vs,
                           point_index=point_index, err=err)
    torch.cuda.synchronize()
    return x, v, vs, int(err.item())


def _mixed(a, b):
    return np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))


def test_fp64_matches_oracle_damped():
    ensure_built()
    n, P, S, seed, k = 777, 200, 600, 13, 3
    w = inputs.josephson_plain(paths=n, steps=S, seed=4)
    x, v, vs, err = _run64(DAMPED, P, S, seed, w["x0"], w["v0"], point_index=k)
    assert err == 0
    xo, vo, so = oracle.jj_run(w["x0"], w["v0"], oracle.jj_params(**DAMPED), P, 0, S, S, seed, point=k)
    ex, ev, es = (_mixed(x.cpu().numpy(), xo), _mixed(v.cpu().numpy(), vo), _mixed(vs.cpu().numpy(), so))
    print("fp64 vs oracle (damped): x %.2e v %.2e vsum %.2e" % (ex, ev, es))
    assert ex <= 1e-11 and ev <= 1e-11 and es <= 1e-10


def _jittered_divergence(point, P, S, seed, x0, v0, steps, realisations=2):
    """How far the FP64 oracle itself moves when every step's state is
    jittered by FP64-rounding-sized relative noise (2e-16): the divergence any
    other FP64 implementation (different cos, log and drive rounding) can be
    expected to show on the same path."""
    rng = np.random.default_rng(77)
    p = oracle.jj_params(**point)
    xo, vo, _ = oracle.jj_run(x0, v0, p, P, 0, steps, S, seed)
    ds = []
    for _ in range(realisations):
        x = np.asarray(x0, np.float64).copy()
        v = np.asarray(v0, np.float64).copy()
        for n in range(steps):
            x, v, _ = oracle.jj_run(x, v, p, P, n, n + 1, S, seed)
            x = x * (1 + 2e-16 * rng.standard_normal(x.size))
            v = v * (1 + 2e-16 * rng.standard_normal(v.size))
        ds.append(np.maximum(np.abs(x - xo) / np.maximum(1, np.abs(xo)), np.abs(v - vo) / np.maximum(1, np.abs(vo))))
    return xo, vo, np.max(ds, axis=0)


def test_fp64_matches_oracle_fig2_sensitivity_gated():
    ensure_built()
    n, P, S, seed = 512, 100, 20_000, 13
    w = inputs.josephson_plain(paths=n, steps=S, seed=4)
    # one drive period: every path within 1e-12
    x, v, _, _ = _run64(FIG2, P, S, seed, w["x0"], w["v0"], 0, 100)
    xo, vo, _ = oracle.jj_run(w["x0"], w["v0"], oracle.jj_params(**FIG2), P, 0, 100, S, seed)
    e100 = max(_mixed(x.cpu().numpy(), xo), _mixed(v.cpu().numpy(), vo))
    assert e100 <= 1e-12
    # ten periods: chaotic growth of rounding differences (Sec. 5); gate each
    # path by the oracle's own divergence d under FP64-sized jitter
    x, v, _, _ = _run64(FIG2, P, S, seed, w["x0"], w["v0"], 0, 1000)
    xo, vo, d = _jittered_divergence(FIG2, P, S, seed, w["x0"], w["v0"], 1000)
    x, v = x.cpu().numpy(), v.cpu().numpy()
    err = np.maximum(np.abs(x - xo) / np.maximum(1, np.abs(xo)), np.abs(v - vo) / np.maximum(1, np.abs(vo)))
    calm = d <= 1e-13
    print("fp64 Fig. 2: 100 steps max err %.2e; 1000 steps max err %.2e, median %.2e vs median d %.2e, "
          "%d calm paths max err %.2e" % (e100, err.max(), np.median(err), np.median(d), calm.sum(),
                                          err[calm].max(initial=0)))
    assert err[calm].max(initial=0) <= 1e-12
    assert np.all(err <= 1e-12 + 100.0 * d)
    assert np.median(err) <= max(np.median(d), 1e-13)


def test_fp64_split_run_is_bit_exact():
    ensure_built()
    n, P, S, seed = 1000, 100, 1000, 2
    w = inputs.josephson_plain(paths=n, steps=S, seed=8)
    a = _run64(FIG2, P, S, seed, w["x0"], w["v0"])
    st = _run64(FIG2, P, S, seed, w["x0"], w["v0"], 0, 437)[:3]
    b = _run64(FIG2, P, S, seed, None, None, 437, S, state=st)
    for u, t in zip(a[:3], b[:3]):
        assert torch.equal(u, t)
    # steps past S are not taken
    c = _run64(FIG2, P, S, seed, None, None, S, S + 50, state=tuple(t.clone() for t in a[:3]))
    assert torch.equal(c[0], a[0]) and torch.equal(c[1], a[1])


def test_fp32_and_fp64_gpu_ensembles_agree_fig2():
    # Sec. 5: the FP32 and FP64 runs of Fig. 2 give the same coarse-grained
    # distribution within its statistical error
    ensure_built()
    n, P, periods, seed = 1 << 16, 100, 200, 31
    S = P * periods
    w = inputs.josephson_plain(paths=n, steps=S, seed=seed)
    ens = sde.Ensemble.josephson([FIG2], [n], [S], seed, steps_per_period=P)
    xg, vg, wg, xf, sg, obs = jj_run(ens, w["x0"], w["v0"], 0, S)
    x64, v64, s64, err = _run64(FIG2, P, S, seed, w["x0"], w["v0"])
    assert err == 0
    x64 = x64.cpu().numpy()
    b32, b64 = np.floor(xg).astype(np.int64), np.floor(x64).astype(np.int64)
    lo, hi = min(b32.min(), b64.min()), max(b32.max(), b64.max())
    c32 = np.bincount(b32 - lo, minlength=hi - lo + 1)
    c64 = np.bincount(b64 - lo, minlength=hi - lo + 1)
    keep = (c32 + c64) >= 10
    table = np.array([np.append(c32[keep], c32[~keep].sum()), np.append(c64[keep], c64[~keep].sum())])
    table = table[:, table.sum(axis=0) > 0]
    chi2, p, dof, _ = stats.chi2_contingency(table)
    # time-averaged velocity over the window: per-path means, FP64 mean and SE
    W = S // 2
    m32, m64 = sg / W, s64.cpu().numpy() / W
    se = np.hypot(m32.std(ddof=1), m64.std(ddof=1)) / np.sqrt(n)
    same = np.mean(b32 == b64)
    print("FP32 vs FP64 on the GPU: %d bins chi2 %.1f dof %d p %.3f; <v> %.6f vs %.6f (SE %.1e); "
          "same period for %.0f%% of paths" % (table.shape[1], chi2, dof, p, m32.mean(), m64.mean(), se,
                                                100 * same))
    assert p > 1e-3
    assert abs(m32.mean() - m64.mean()) <= 3 * se
    assert abs(obs["mean"][0] - m32.mean()) <= 1e-9 * max(1.0, abs(m32.mean()))


def test_fp64_invalid_arguments_and_nonfinite():
    ensure_built()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    v = torch.zeros_like(x)
    with pytest.raises(sde.SDEError):
        sde.josephson_run_fp64(FIG2, 0, 10, 1, 0, 10, x, v, x, v)
    with pytest.raises(sde.SDEError):
        sde.josephson_run_fp64(dict(FIG2, omega=-1.0), 100, 10, 1, 0, 10, x, v, x, v)
    with pytest.raises(sde.SDEError):
        sde.josephson_run_fp64(FIG2, 100, 10, 1, 5, 4, x, v, x, v)
    # a state that overflows: the error word gets the non-finite bit
    x2, v2, _, err = _run64(dict(FIG2, gamma=1e300), 100, 20, 1, np.zeros(8), np.ones(8))
    assert err == 1
