"""The allocation-free entry point (sde_josephson_run_noalloc) against the
regular one (sde_create + sde_run_ensemble, plain schedule, one path per
thread), through the C ABI, on two calls in a row.

It exists for callers that may not allocate device memory (another
framework's memory pool, a stream being captured into a CUDA graph, hosts
that reserve all device memory up front); its scratch is a fixed static array
shared by every call, so the second call checks that what the first call left
there does no harm.  This file is collected last so that a failure here stops
a -x run only after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import ensure_built, jj_run, mixed_rel
from paper_0903_3852_gb300 import inputs, sde

pytestmark = pytest.mark.gpu

P = 200


def _noalloc(point, n, S, seed, x0, v0, n_end):
    dev = torch.device("cuda")
    x_in = torch.from_numpy(np.ascontiguousarray(x0, np.float32)).to(dev)
    v_in = torch.from_numpy(np.ascontiguousarray(v0, np.float32)).to(dev)
    x_out, v_out = torch.empty_like(x_in), torch.empty_like(v_in)
    w_out = torch.empty(n, dtype=torch.int32, device=dev)
    s_out = torch.empty(n, dtype=torch.float64, device=dev)
    obs = torch.full((5,), float("nan"), dtype=torch.float64, device=dev)
    sde.josephson_run_noalloc(point, P, n, S, seed, 0, n_end, x_in, v_in, x_out, v_out, w_out, s_out, obs)
    torch.cuda.synchronize()
    x = w_out.cpu().numpy().astype(np.float64) + x_out.cpu().numpy().astype(np.float64)
    return x, v_out.cpu().numpy().astype(np.float64), s_out.cpu().numpy(), obs.cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice():
    ensure_built()
    cases = [
        # (point, paths, total steps, seed): the second call is smaller, with
        # another seed, so stale partials of the first would show up
        (dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3), 1000, 3000, 7),
        (dict(gamma=3.0, a=1.0, omega=2.0, f=0.3, D=1e-2), 333, 2001, 11),
    ]
    for point, n, S, seed in cases:
        w = inputs.josephson_custom([point], [n], [S], seed=seed)
        ens = sde.Ensemble.josephson([point], [n], [S], seed, steps_per_period=P,
                                     schedule=sde.SDE_SCHED_PLAIN, block_threads=256, paths_per_thread=1)
        xr, vr, _, _, sr, obs_r = jj_run(ens, w["x0"], w["v0"], 0, S)
        ens.close()
        xa, va, sa, obs_a = _noalloc(point, n, S, seed, w["x0"], w["v0"], S)
        # same arithmetic on both sides; held to the parity tolerance of the suite
        assert mixed_rel(xa, xr).max() <= 1e-5
        assert mixed_rel(va, vr).max() <= 1e-5
        assert np.max(np.abs(sa - sr) / np.maximum(1.0, np.abs(sr))) <= 1e-5
        row = obs_r[0]
        assert obs_a[3] == row["count"] == n
        assert abs(obs_a[0] - row["mean"]) <= 1e-5 * max(1.0, abs(row["mean"]))
        assert abs(obs_a[2] - row["se"]) <= 1e-5 * max(1.0, abs(row["se"]))
        assert abs(obs_a[4] - row["t"]) <= 1e-12 * row["t"]


def test_noalloc_rejects_sizes_beyond_its_array():
    """The C entry point itself refuses more paths than its static array covers,
    before it touches any buffer (called through ctypes directly: the Python
    wrapper would already refuse the undersized buffers passed here)."""
    L = ensure_built()
    p = sde.JJPoint(0.9, 4.2, 4.9, 0.1, 1e-3)
    t = torch.empty(1, device="cuda")
    obs = torch.empty(5, dtype=torch.float64, device="cuda")
    ptr = t.data_ptr()
    st = L.sde_josephson_run_noalloc(ctypes.byref(p), P, sde.NOALLOC_MAX_PATHS + 1, 10, 0, 0, 10,
                                     ptr, ptr, None, None, ptr, ptr, ptr, ptr, obs.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == sde.SDE_ERR_INVALID_ARG
    assert "at most" in L.sde_last_error().decode()
