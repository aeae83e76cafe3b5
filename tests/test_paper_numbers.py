"""The paper's printed operation counts, workload sizes and run times
(tests/golden/paper_numbers.txt) against the FLOP models, workloads and
reference rates the benchmark uses."""
import math
import os

import pytest

import bench
from paper_0903_3852_gb300 import inputs


@pytest.fixture(scope="module")
def paper(golden_dir):
    rows = {}
    table1 = []
    with open(os.path.join(golden_dir, "paper_numbers.txt")) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "table1":
                table1.append((int(vals[0]), vals[1], int(vals[2])))
            elif key == "ops":
                rows[("ops", vals[0])] = [int(v) for v in vals[1:]]
            elif key.endswith("_params"):
                rows[key] = {vals[i]: float(vals[i + 1]) for i in range(0, len(vals), 2)}
            else:
                rows[key] = [float(v) for v in vals]
    rows["table1"] = table1
    return rows


def test_table1_weights_sum_to_its_total_and_the_bench_model(paper):
    total = sum(count * weight for count, _, weight in paper["table1"])
    assert total == paper["table1_total"][0] == 79
    assert paper[("ops", "prog1")] == [total]
    assert bench.PAPER_FLOP_PER_STEP == total


def test_kuramoto_operation_counts_are_the_bench_models(paper):
    assert bench.PAPER_FLOP_MEANFIELD == paper[("ops", "prog3")][0]
    base, per_pair = paper[("ops", "prog2")]
    assert (base, bench.PAPER_FLOP_PAIR) == (44, per_pair)


def test_prog1_rate_times_table1_is_the_printed_gflops(paper):
    # the 79 FLOP are per time step of one path: the unit of path-steps/s
    gflops = paper["prog1_rate"][0] * paper["table1_total"][0] / 1e9
    assert abs(gflops - paper["prog1_gflops"][0]) <= 0.01 * paper["prog1_gflops"][0]


def test_fig2_workload_and_reference_rates(paper):
    w = inputs.josephson_fig2()
    paths = int(paper["fig2_paths"][0])
    steps = round(paper["fig2_periods"][0] / paper["fig2_dt_per_period"][0])
    assert int(w["paths"][0]) == paths == 2 ** 19
    assert int(w["steps"][0]) == steps == 200_000
    assert w["steps_per_period"] == round(1.0 / paper["fig2_dt_per_period"][0])
    pt = w["points"][0]
    for k, v in paper["fig2_params"].items():
        assert math.isclose(pt[k], v)
    fp32_s, fp64_s = paper["fig2_seconds"]
    assert math.isclose(bench.PAPER_RATE["fig2"], paths * steps / fp32_s)
    assert math.isclose(bench.PAPER_RATE["fig2-fp64"], paths * steps / fp64_s)


def test_fig4_workload(paper):
    w = inputs.kuramoto_fig4()
    assert w["n_osc"] * w["replicas"] == int(paper["fig4_oscillators"][0]) == 2 ** 24
    prm = paper["fig4_params"]
    assert (w["omega"] == prm["omega"]).all()
    assert w["K"] == prm["K"] and w["D"] == prm["T"]  # T: the noise intensity of Eq. 2
