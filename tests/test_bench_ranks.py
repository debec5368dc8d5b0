"""Host logic of bench.py on CPU: two gloo ranks agree on the
slowest rank's time, the job value counts every rank's replica, the
reference arm runs on rank 0 only and prints the contract's JSON line, and
the clock record of the timed region is read from nvidia-smi's lines."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        q.put((rank, ms, bench.job_value(world, 1000, 4, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, value in got:
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.015)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 10, 2, 1000.0) == pytest.approx(20.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 1, 2

    assert bench.run_reference(Args()) == 0
    assert capsys.readouterr().out == ""


def test_clock_summary_reads_nvidia_smi_lines():
    """The clock record of the timed region: the median SM clock under load,
    the maximum, and every throttle reason seen Active at least once
    (nvidia-smi --format=csv,noheader,nounits lines of the bench's query)."""
    c = bench.ClockSampler(None)
    c.out = "\n".join([
        "2070, 2070, 910.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1390.20, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "1980, 2070, 1401.00, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "[N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ])
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.out = "1200, 2070, 700.0, 0x0000000000000008, Not Active, Active, Not Active, Not Active\n"
    assert c.summary()["reasons"] == ["hw_thermal_slowdown"]
    c.out = ""
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the CPU oracle on a bounded sample) prints
    one JSON line with the keys of the bench contract, its own cpu_baseline
    and an e2e block that moves no bytes."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] >= 3 and d["n_gpus"] == 1
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOAD
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"] and d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == 2
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
