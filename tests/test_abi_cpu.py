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
    assert L.sde_abi_version() == 100
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
