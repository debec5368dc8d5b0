"""The committed bench line (profiles/bench_line_bubble3d.json, written by a
`python bench.py` run on a GB300) against the bench contract and against
bench.py's own byte counts: every key the contract asks for is there, and the
derived numbers agree with the measured ones they come from (the value with
the step time and the grid, the roofline fraction with its rate and peak, the
algorithmic bytes with the per-cell word counts of the 3D step, and in the
batch, axisymmetric, static-drop and surrogate sections each rate, speedup,
Laplace ratio, bar verdict and forward roofline with its own inputs)."""
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


def test_the_batch_axisymmetric_and_static_drop_sections(line):
    from paper_2011_00814_gb300 import inputs
    b = line["batch2d"]
    prms, _ = inputs.batch_instances(n=96, seed=0, precision=32)
    assert b["cells"] == sum(p["nx"] * p["ny"] for p in prms)
    for arm in ("batched", "loop"):
        assert close(b[arm]["cell_updates_per_s"] * b[arm]["ms_per_step"] / 1e3, b["cells"])
    assert close(b["speedup"], b["batched"]["cell_updates_per_s"] / b["loop"]["cell_updates_per_s"])
    # 49 words (196 B) per 2D cell-update with TVD-RK2 CH
    assert close(b["step_algorithmic_gbs"], 49 * 4 * b["batched"]["cell_updates_per_s"] / 1e9)
    assert close(b["step_frac"], b["step_algorithmic_gbs"] / line["roofline"]["peak"])
    a = line["axisym"]
    assert a["cells"] == 400 * 1200
    for prec in ("fp32", "fp64"):
        assert close(a[prec]["cell_updates_per_s"] * a[prec]["ms_per_step"] / 1e3, a["cells"])
        assert a[prec]["nan"] == 0
    sd = line["static_drop"]
    for r in (sd["advective"], sd["advective"]["settled"]):
        assert close(r["sigma_over_R_eff"] * r["R_eff"], sd["advective"]["sigma_over_R_eff"] * sd["advective"]["R_eff"])
        assert close(r["dP_over_laplace"], r["dP"] / r["sigma_over_R_eff"])
        assert close(r["dp_over_laplace"], r["dp"] / r["sigma_over_R_eff"])
        assert r["within_2pct"] == (abs(r["dP_over_laplace"] - 1.0) <= 0.02)
    for form in ("advective", "conservative"):
        r = sd[form]
        assert close(r["max_spurious_u_over_Uc"], r["max_spurious_u"] / sd["U_c"])
    assert sd["conservative"]["int_phi_drift"] == 0.0


def test_the_surrogate_section(line):
    s = line["surrogate"]
    bars = s["bars"]
    for key in ("network", "persistence"):
        rs = [c[key] for c in s["cases"]]
        for r in rs:
            assert close(r["speedup"], r["solver_ms"] / r["controller_ms"])
            assert r["meets_bars"] == (r["phi_l2"] <= bars["phi_l2"] and r["interface_max"] <= bars["interface_cells"])
            st = r["stats"]
            assert st["calls"] == 64 and st["net_calls"] <= st["calls"] and st["failures"] <= st["checks"]
        summ = s[key]
        assert close(summ["speedup"], sum(r["speedup"] for r in rs) / len(rs))
        assert summ["phi_l2_max"] == max(r["phi_l2"] for r in rs)
        assert summ["interface_max_cells"] == max(r["interface_max"] for r in rs)
        assert summ["check_failures"] == sum(r["stats"]["failures"] for r in rs)
        assert summ["meets_bars_every_case"] == all(r["meets_bars"] for r in rs)
    # the speedup is claimed only for a configuration that meets both bars on every case
    if s["network"]["meets_bars_every_case"]:
        assert s["speedup_at_tolerance"] == s["network"]["speedup"]
    else:
        assert s["speedup_at_tolerance"] is None
    f8, f1 = s["forward"], s["forward_batch1"]
    assert f8["batch"] == 8 and f1["batch"] == 1 and close(f8["gflop"], 8 * f1["gflop"])
    for f in (f8, f1):
        r = f["roofline"]
        assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
        assert close(r["achieved"], f["gflop"] / (f["ms"] / 1e3) / 1e3)
        assert close(r["frac"], r["achieved"] / r["peak"]) and 0 < r["frac"] < 1.05


def test_the_stored_dram_traffic_is_the_capture_scaled_to_the_grid(line):
    with open(os.path.join(HERE, "..", "profiles", "flow_stage_bubble3d_traffic.json")) as f:
        t = json.load(f)
    per = [t[s]["dram_bytes_read"] + t[s]["dram_bytes_write"] for s in ("stage2", "stage3")]
    assert close(t["bytes_per_launch_captured"], sum(per) / 2)
    # captured on 128 x 128 x 256, scaled by cells to 256 x 256 x 512
    assert t["scale_to_full_grid"] == (256 * 256 * 512) / (128 * 128 * 256)
    assert close(t["bytes_per_launch_full_grid"], t["bytes_per_launch_captured"] * t["scale_to_full_grid"])
    w = (t["stage2"]["algorithmic_bytes_per_cell"] + t["stage3"]["algorithmic_bytes_per_cell"]) / 2
    assert w == (bench.WORDS["flow_stage2"] + bench.WORDS["flow_stage3"]) / 2 * 4
    assert close(t["algorithmic_bytes_per_launch_full_grid"], w * 256 * 256 * 512)
    assert t["command"].startswith("ncu ") and "--clock-control none" in t["command"]
    # the bench line carries this figure when its kernel sources were those of the capture
    if line["roofline"]["traffic"] is not None:
        assert close(line["roofline"]["traffic"], t["bytes_per_launch_full_grid"])
