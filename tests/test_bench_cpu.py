"""Host logic of the benchmark (no GPU): the reference arm (the oracle on the
host cores) reports the same workload, by name and size, as the GPU arm."""
import sys

import numpy as np

import bench
from paper_0903_3852_gb300 import inputs


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_reference_config_names_the_gpu_arms_workload():
    w = inputs.josephson_sweep()
    cfg = bench.reference_config(_args(), "sample")
    assert cfg["workload"] == "josephson_sweep_512pts"
    assert cfg["points"] == 512 and cfg["total_paths"] == int(w["paths"].sum())
    assert cfg["path_steps"] == float((w["paths"] * w["steps"]).sum())
    assert cfg["steps_per_period"] == 200 and cfg["sample"] == "sample"
    assert bench.reference_config(_args("--workload", "fig2"), "s")["workload"] == \
        "josephson_fig2_524288paths_2e5steps"
    assert bench.reference_config(_args("--workload", "plain"), "s")["workload"] == "josephson_plain_1024"
    capped = bench.reference_config(_args("--steps-cap", "2000", "--euler"), "s")
    assert capped["workload"] == "josephson_sweep_512pts_cap2000_euler"
    assert capped["path_steps"] == float(np.minimum(w["steps"], 2000).dot(w["paths"]))


def test_reference_config_names_the_kuramoto_workloads():
    names = {w: bench.reference_config(_args("--workload", w), "s")["workload"]
             for w in ("kuramoto-meanfield", "kuramoto-pairwise", "kuramoto-fig4", "kuramoto-general",
                       "kuramoto-general-fp32")}
    assert names == {"kuramoto-meanfield": "kuramoto_meanfield_N4096_R64",
                     "kuramoto-pairwise": "kuramoto_pairwise_N4096_R64",
                     "kuramoto-fig4": "kuramoto_fig4_meanfield_grid_N16777216_R1",
                     "kuramoto-general": "kuramoto_general_bf16_tcgen05_N8192_R256",
                     "kuramoto-general-fp32": "kuramoto_general_fp32_cudacore_N8192_R256"}
    assert bench.reference_config(_args("--workload", "kuramoto-pairwise", "--euler"), "s")["workload"] == \
        "kuramoto_pairwise_N4096_R64_euler_prog2"
