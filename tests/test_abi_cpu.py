"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function include/sde.h declares, the ctypes structures match the C
layout, and argument validation that happens before any CUDA call."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_0903_3852_gb300 import build as sde_build
from paper_0903_3852_gb300 import sde

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sde.h")


@pytest.fixture(scope="module")
def L():
    sde_build.build()
    return sde.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[a-zA-Z_][\w\s\*]*?\b(sde_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sde_create", "sde_run_ensemble", "sde_observables", "sde_destroy",
                     "sde_philox4x32_10", "sde_box_muller"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    out = subprocess.run(["nm", "-D", "--defined-only", sde.LIB_PATH], stdout=subprocess.PIPE,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    bound = {s[0] for s in sde.SIGNATURES}
    assert set(declared_functions()) <= bound | {"sde_last_error"}


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "sde.h"
#define F(T, m) printf(#T "." #m " %zu\n", offsetof(T, m))
int main(void) {
  printf("sde_config %zu\nsde_run_desc %zu\nsde_obs_row %zu\nsde_jj_point %zu\n",
         sizeof(sde_config), sizeof(sde_run_desc), sizeof(sde_obs_row), sizeof(sde_jj_point));
  F(sde_config, seed); F(sde_config, points); F(sde_config, n_osc); F(sde_config, dt);
  F(sde_config, sample_every); F(sde_config, flags); F(sde_config, cluster_ctas);
  F(sde_run_desc, r_out_dev); F(sde_run_desc, vsum_out_dev);
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    lines = dict(l.rsplit(" ", 1) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    assert int(lines["sde_config"]) == ctypes.sizeof(sde.Config)
    assert int(lines["sde_run_desc"]) == ctypes.sizeof(sde.RunDesc)
    assert int(lines["sde_obs_row"]) == ctypes.sizeof(sde.ObsRow)
    assert int(lines["sde_jj_point"]) == ctypes.sizeof(sde.JJPoint)
    for key, val in lines.items():
        if "." in key:
            struct, field = key.split(".")
            cls = {"sde_config": sde.Config, "sde_run_desc": sde.RunDesc}[struct]
            assert getattr(cls, field).offset == int(val), key


def test_validation_before_any_cuda_call(L):
    assert L.sde_abi_version() == 102
    h = ctypes.c_void_p()
    assert L.sde_create(None, ctypes.byref(h)) == 1
    assert b"cfg" in L.sde_last_error()
    assert L.sde_create(None, None) == 1
    assert L.sde_philox4x32_10(None, 0, None, -1, None) == 1
    assert L.sde_box_muller(None, 0, None, 5, None) == 1
    assert L.sde_run_ensemble(None, None, None) == 1
    assert L.sde_observables(None, None, 0, None) == 1
    assert L.sde_josephson_run_fp64(None, 100, 8, 10, 1, 0, 0, 10, None, None, None, None, None, None, None,
                                    None) == 1
    pt = sde.JJPoint(0.9, 4.2, 4.9, 0.1, 1e-3)
    assert L.sde_josephson_run_fp64(ctypes.byref(pt), 0, 8, 10, 1, 0, 0, 10, None, None, None, None, None, None,
                                    None, None) == 1
    assert b"steps_per_period" in L.sde_last_error()
    assert L.sde_josephson_run_fp64(ctypes.byref(pt), 100, 0, 10, 1, 0, 0, 10, None, None, None, None, None,
                                    None, None, None) == 0  # no paths: nothing to do
    L.sde_destroy(None)  # NULL-safe


FIG2 = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)


def _create_status(make):
    """Status of sde_create for a configuration built by `make` (0 if created)."""
    try:
        e = make()
    except sde.SDEError as err:
        return err.status, str(err)
    del e
    return sde.SDE_OK, ""


@pytest.mark.parametrize("kw,field", [
    (dict(points=[], paths=[], steps=[]), "n_points"),
    (dict(steps_per_period=0), "steps_per_period"),
    (dict(steps_per_period=4097), "steps_per_period"),
    (dict(schedule=7), "schedule"),
    (dict(block_threads=48), "block_threads"),
    (dict(block_threads=1024), "block_threads"),
    (dict(paths_per_thread=3), "paths_per_thread"),
    (dict(paths_per_thread=24), "paths_per_thread"),
    (dict(points=[dict(FIG2, omega=0.0)]), "omega"),
    (dict(points=[dict(FIG2, gamma=-1.0)]), "gamma"),
    (dict(points=[dict(FIG2, D=-1e-3)]), "D"),
    (dict(points=[dict(FIG2, a=float("nan"))]), "finite"),
    (dict(paths=[-1]), "paths"),
    (dict(steps=[(1 << 33) + 1]), "steps"),
])
def test_josephson_config_is_checked_before_any_cuda_call(L, kw, field):
    # the checks run on the host first, so they answer the same with or
    # without a GPU
    args = dict(points=[FIG2], paths=[64], steps=[100], steps_per_period=200)
    args.update(kw)
    pts, paths, steps, P = args.pop("points"), args.pop("paths"), args.pop("steps"), args.pop("steps_per_period")
    status, msg = _create_status(lambda: sde.Ensemble.josephson(pts, paths, steps, 0, steps_per_period=P, **args))
    assert status == sde.SDE_ERR_INVALID_ARG and field in msg, (status, msg)


@pytest.mark.parametrize("kw,status,field", [
    (dict(n_osc=0), sde.SDE_ERR_INVALID_ARG, "n_osc"),
    (dict(n_replicas=0), sde.SDE_ERR_INVALID_ARG, "n_replicas"),
    (dict(dt=0.0), sde.SDE_ERR_INVALID_ARG, "dt"),
    (dict(D=-0.1), sde.SDE_ERR_INVALID_ARG, "D"),
    (dict(K=float("inf")), sde.SDE_ERR_INVALID_ARG, "finite"),
    (dict(flags=sde.SDE_FLAG_EULER), sde.SDE_ERR_UNSUPPORTED, "Euler"),
    (dict(schedule=sde.SDE_SCHED_GRID, cluster_ctas=2), sde.SDE_ERR_INVALID_ARG, "grid-wide"),
])
def test_kuramoto_config_is_checked_before_any_cuda_call(L, kw, status, field):
    args = dict(n_osc=1024, n_replicas=4, K=2.0, D=0.05, dt=0.01)
    args.update(kw)
    got, msg = _create_status(lambda: sde.Ensemble.kuramoto(
        sde.SDE_KURAMOTO_MEANFIELD, args.pop("n_osc"), args.pop("n_replicas"), args.pop("K"), args.pop("D"),
        args.pop("dt"), 0, **args))
    assert got == status and field in msg, (got, msg)


def test_valid_configs_pass_the_host_checks(L):
    # a valid configuration gets past validation: with a GPU it is created,
    # without one the first CUDA call fails instead
    ok = (sde.SDE_OK, sde.SDE_ERR_CUDA)
    st, msg = _create_status(lambda: sde.Ensemble.josephson([FIG2], [64], [100], 0, steps_per_period=200,
                                                            paths_per_thread=14))
    assert st in ok, msg
    st, msg = _create_status(lambda: sde.Ensemble.kuramoto(sde.SDE_KURAMOTO_PAIRWISE, 1024, 4, 2.0, 0.05, 0.01, 0,
                                                           flags=sde.SDE_FLAG_EULER))
    assert st in ok, msg


def test_noalloc_wrapper_checks_buffers_before_the_call():
    """sde_josephson_run_noalloc sees bare pointers, so its binding checks every
    buffer's length, dtype and device first: a short or mistyped buffer raises
    on the host and nothing is launched (CPU tensors: no GPU involved)."""
    import torch
    pt = dict(gamma=0.9, a=4.2, omega=4.9, f=0.1, D=1e-3)
    n = 64
    f32 = lambda k: torch.zeros(k, dtype=torch.float32)  # noqa: E731
    good = dict(x_in=f32(n), v_in=f32(n), x_out=f32(n), v_out=f32(n),
                w_out=torch.zeros(n, dtype=torch.int32), vsum_out=torch.zeros(n, dtype=torch.float64),
                obs_out=torch.zeros(5, dtype=torch.float64))

    def call(**over):
        b = dict(good, **over)
        sde.josephson_run_noalloc(pt, 200, n, 100, 0, 0, 100, b["x_in"], b["v_in"], b["x_out"], b["v_out"],
                                  b["w_out"], b["vsum_out"], b["obs_out"], w_in=b.get("w_in"),
                                  vsum_in=b.get("vsum_in"))

    with pytest.raises(ValueError, match="fewer than"):
        call(v_out=f32(n - 1))
    with pytest.raises(ValueError, match="fewer than"):
        call(vsum_in=torch.zeros(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="must be torch.int32"):
        call(w_out=torch.zeros(n, dtype=torch.int64))
    with pytest.raises(ValueError, match="must be torch.float64"):
        call(vsum_out=torch.zeros(n, dtype=torch.float32))
    with pytest.raises(ValueError, match="fewer than"):
        call(obs_out=torch.zeros(4, dtype=torch.float64))
    # right sizes and types, but host memory: refused before the C call
    with pytest.raises(ValueError, match="current CUDA device"):
        call()


def test_injected_allocation_failure_reports_no_memory(L):
    """sde_debug_fail_allocation(1) makes the next sde_create fail at its first
    allocation, the host context, after validation and before any CUDA call:
    SDE_ERR_NO_MEMORY and a NULL context; the injection is then disarmed."""
    pts = (sde.JJPoint * 1)(sde.JJPoint(0.9, 4.2, 4.9, 0.1, 1e-3))
    paths = (ctypes.c_int64 * 1)(64)
    steps = (ctypes.c_int64 * 1)(100)
    cfg = sde.Config()
    cfg.model, cfg.schedule, cfg.n_points, cfg.steps_per_period = sde.SDE_JOSEPHSON, 0, 1, 200
    cfg.points = ctypes.cast(pts, ctypes.POINTER(sde.JJPoint))
    cfg.paths, cfg.steps = paths, steps
    cfg.block_threads, cfg.paths_per_thread = 128, 1
    h = ctypes.c_void_p(1)
    L.sde_debug_fail_allocation(1)
    assert L.sde_create(ctypes.byref(cfg), ctypes.byref(h)) == sde.SDE_ERR_NO_MEMORY
    assert h.value is None
    assert "allocation" in L.sde_last_error().decode()
    # disarmed: the next call gets past the host allocation (without a GPU it
    # then stops at the first CUDA call)
    st = L.sde_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st != sde.SDE_ERR_NO_MEMORY
    if st == sde.SDE_OK:
        L.sde_destroy(h)
    assert L.sde_set_wait_limit(None, 5) == sde.SDE_ERR_INVALID_ARG


def test_binding_constants_equal_the_header(tmp_path):
    # every status, model, schedule and flag the binding names, printed by a C
    # program compiled against include/sde.h
    names = [n for n in dir(sde) if n.startswith("SDE_") and isinstance(getattr(sde, n), int)]
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "sde.h"\nint main(void) {\n'
                   + "".join('  printf("%s %%lld\\n", (long long)(%s));\n' % (n, n) for n in names)
                   + '  printf("SDE_NOALLOC_MAX_PATHS %lld\\n", (long long)SDE_NOALLOC_MAX_PATHS);\n'
                   + "  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).split("\n") if l)
    assert len(names) >= 20
    for n in names:
        assert int(got[n]) == getattr(sde, n), n
    assert int(got["SDE_NOALLOC_MAX_PATHS"]) == sde.NOALLOC_MAX_PATHS
    flags = [getattr(sde, n) for n in names if n.startswith("SDE_FLAG_")]
    assert all(f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)  # distinct single bits
