"""The committed bench line (profiles/bench_line_bubble3d.json, written by a
`python bench.py` run on a GB300) against the bench contract and against
bench.py's own byte counts: every key the contract asks for is there, and the
derived numbers agree with the measured ones they come from (the value with
the step time and the grid, the roofline fraction with its rate and peak, the
algorithmic bytes with the per-cell word counts of the 3D step)."""
import json
import math
import os

import pytest

import bench

HERE = os.path.dirname(os.path.abspath(__file__))
LINE = os.path.join(HERE, "..", "profiles", "bench_line_bubble3d.json")

# flow stages 1-3, CH stages 1-4 (RK4), mu after each CH stage
LAUNCHES_PER_STEP = 3 + 4 + 4


@pytest.fixture(scope="module")
def line():
    with open(LINE) as f:
        return json.load(f)


def close(a, b, rel=1e-9):
    return math.isclose(a, b, rel_tol=rel)


def test_the_contract_keys_are_there(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in line, k
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["config"]["workload"] == bench.WORKLOAD
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["data"] == "synthetic"
    assert line["dtype"] == "f32" and line["vs_baseline"] is None
    assert line["warmup"] >= 3 and line["steps"] >= 1 and line["n_gpus"] >= 1
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"], k
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in line["clocks"], k


def test_the_value_is_the_grid_over_the_step_time(line):
    cells = line["config"]["cells"]
    assert cells == 256 * 256 * 512
    # value = n_gpus * cells * steps / (steps * ms_per_step / 1000)
    assert close(line["value"] * line["ms_per_step"] / 1e3, line["n_gpus"] * cells)


def test_the_roofline_follows_from_its_rate_and_peak(line):
    r = line["roofline"]
    cells = line["config"]["cells"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_kind"] == "measured"
    assert close(r["frac"], r["achieved"] / r["peak"])
    assert close(r["gap_to_target"], r["target_frac"] - r["frac"])
    # the mean algorithmic bytes of flow stages 2 and 3 per launch
    w = (bench.WORDS["flow_stage2"] + bench.WORDS["flow_stage3"]) / 2
    assert close(r["algorithmic_bytes_per_launch"], w * 4 * cells)
    # the whole step's algorithmic bytes over the measured step time
    words = (bench.WORDS["flow_stage1"] + bench.WORDS["flow_stage2"] + bench.WORDS["flow_stage3"]
             + sum(bench.CH_WORDS_RK4) + 4 * bench.WORDS["mu"])
    assert close(r["step_algorithmic_gbs"], words * 4 * cells / (line["ms_per_step"] / 1e3) / 1e9)
    assert close(r["step_frac"], r["step_algorithmic_gbs"] / r["peak"])
    # a fraction above 1 would mean the timed kernel does not do the work counted
    assert 0 < r["frac"] < 1.05 and 0 < r["step_frac"] < 1.05
    # DRAM traffic (ncu) is at least the algorithmic bytes and not far above them
    if r["traffic"] is not None:
        assert 0.95 <= r["traffic"] / r["algorithmic_bytes_per_launch"] <= 1.5
    assert abs(sum(r["shares"].values()) - 1.0) < 1e-3


def test_the_end_to_end_copies_and_launch_count(line):
    cells = line["config"]["cells"]
    e = line["e2e"]
    assert e["unit"] == line["unit"]
    # five FP64 fields (phi, u, v, w, p) in and out every step
    assert e["h2d_bytes_per_step"] == 5 * 8 * cells and e["d2h_bytes_per_step"] == 5 * 8 * cells
    # the host link bounds e2e below the device-resident value
    assert 0 < e["value"] < line["value"]
    assert line["gpu_launches"] == LAUNCHES_PER_STEP * line["steps"]


def test_the_clock_record_is_clean(line):
    c = line["clocks"]
    for bad in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bad not in c["reasons"]
    assert c["sm_mhz"] >= 0.9 * c["sm_max_mhz"]
