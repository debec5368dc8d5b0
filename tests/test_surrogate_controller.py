"""The surrogate controller's decisions, on the CPU with stand-ins for the
network and the solver.

The controller (a check every ``check_every`` calls against K solver steps
from the same start, roll-back to the last verified state and recomputation
by the solver when the check fails, then ``cooldown`` windows on the solver
alone) is host logic.  Here the state is two numbers, the time t in steps and
a "drift" that only the network adds; the solver advances t exactly and adds
nothing.  So after every call t must equal calls * K, and the drift tells
which network results were kept.

The calibration of the check's displacement tolerance is host logic too: with
a stand-in for the solver comparison it must keep the largest candidate at
which every case ends within the margin of both bars.
"""
from __future__ import annotations

import math
import types

import numpy as np
import pytest

from paper_2011_00814_gb300 import surrogate

K = 64
DISP_PER_DRIFT = 100.0


class FakeSolver:
    def __init__(self):
        self.t, self.drift = 0, 0.0
        self.advanced = 0

    def pack(self, buf):
        buf.flat[0], buf.flat[1] = self.t, self.drift

    def unpack(self, buf):
        self.t, self.drift = int(buf.flat[0]), float(buf.flat[1])

    def advance(self, n):
        self.t += n
        self.advanced += n

    def distance(self, buf):
        # relative phi-L2-like distance between buf's state and the solver's
        if int(buf.flat[0]) != self.t:
            return (1e300, 1.0)
        return ((float(buf.flat[1]) - self.drift) ** 2, 1.0)

    def interface_distance(self, buf):
        # interface displacement in cells: DISP_PER_DRIFT cells per unit of drift
        if int(buf.flat[0]) != self.t:
            return (math.inf, math.inf)
        d = abs(float(buf.flat[1]) - self.drift) * DISP_PER_DRIFT
        return (d, d)


class FakeNet:
    """Advances the packed state by K steps and adds errs[i] on its i-th call."""

    check_tol, check_tol_disp = 2e-2, 1.0

    def __init__(self, errs):
        self.K, self.n = K, 2
        self.errs = list(errs)
        self.calls = 0

    def forward(self, x, y, batch):
        y.flat[0] = x.flat[0] + K
        y.flat[1] = x.flat[1] + self.errs[self.calls]
        self.calls += 1


@pytest.fixture
def numpy_buffers(monkeypatch):
    fake = types.SimpleNamespace(float32=np.float32,
                                 empty=lambda shape, dtype=None, device=None: np.zeros(shape),
                                 empty_like=lambda a: np.zeros_like(a))
    monkeypatch.setattr(surrogate, "_torch", lambda: fake)


def _run(errs, calls, **kw):
    net, sol = FakeNet(errs), FakeSolver()
    c = surrogate.Controller(net, sol, **kw)
    for i in range(calls):
        c.call()
        assert sol.t == (i + 1) * K, i          # time bookkeeping holds on every path
    return c.stats, sol, net


def test_all_checks_pass(numpy_buffers):
    errs = [1e-3] * 16
    st, sol, net = _run(errs, 16, check_every=4, tol=2e-2)
    assert (st.calls, st.net_calls, st.checks, st.failures) == (16, 16, 4, 0)
    assert st.solver_calls == 4
    # every window keeps three network results; the fourth is replaced by the solver's
    assert sol.drift == pytest.approx(4 * 3 * 1e-3)
    assert st.check_l2 == pytest.approx([1e-3] * 4)


def test_failed_check_rolls_back_and_cools_down(numpy_buffers):
    # window 1 passes; window 2's check fails (error 0.05 on its fourth call),
    # so it is recomputed by the solver from the state after window 1, and
    # window 3 (cooldown 1) runs on the solver alone; window 4 uses the network
    errs = [1e-3] * 7 + [5e-2] + [2e-3] * 4
    st, sol, net = _run(errs, 16, check_every=4, tol=2e-2, cooldown=1)
    assert st.checks == 3 and st.failures == 1
    assert st.net_calls == 12 and net.calls == 12
    # solver K-step runs: 3 checks, 4 to recompute window 2, 4 in cooldown
    assert st.solver_calls == 3 + 4 + 4
    assert sol.advanced == st.solver_calls * K
    # kept: three network results of window 1 and three of window 4
    assert sol.drift == pytest.approx(3 * 1e-3 + 3 * 2e-3)
    assert st.max_check_l2 == pytest.approx(5e-2)


def test_interface_displacement_alone_fails_a_check(numpy_buffers):
    # every check's phi error (1e-2) is within tol = 2e-2, but its interface
    # displacement (1 cell) exceeds tol_disp = 0.5: each check fails, its
    # window is recomputed by the solver and none of the network's results is kept
    errs = [0.0, 0.0, 0.0, 1e-2] * 2
    st, sol, net = _run(errs, 12, check_every=4, tol=2e-2, tol_disp=0.5, cooldown=1)
    assert st.checks == 2 and st.failures == 2
    assert st.check_l2 == pytest.approx([1e-2, 1e-2])
    assert st.check_disp == pytest.approx([1.0, 1.0])
    assert sol.drift == 0.0
    # the same run with the displacement tolerance at 2 cells keeps every window
    st, sol, net = _run(errs + [0.0] * 4, 12, check_every=4, tol=2e-2, tol_disp=2.0, cooldown=1)
    assert st.failures == 0 and st.checks == 3


def test_defaults_come_from_the_surrogate(numpy_buffers):
    net, sol = FakeNet([0.0] * 4), FakeSolver()
    c = surrogate.Controller(net, sol)
    assert (c.tol, c.tol_disp) == (FakeNet.check_tol, FakeNet.check_tol_disp)


def test_nan_check_counts_as_a_failure(numpy_buffers):
    errs = [0.0, 0.0, 0.0, math.nan]
    st, sol, net = _run(errs, 4, check_every=4, tol=2e-2)
    assert st.failures == 1 and sol.drift == 0.0


def test_persistence_baseline_never_calls_the_network(numpy_buffers):
    net, sol = FakeNet([]), FakeSolver()
    c = surrogate.Controller(net, sol, check_every=4, tol=2e-2, persistence=True)
    c.call()
    # persistence leaves the state where it was: the call falls behind the
    # solver's clock, which the first check catches
    assert net.calls == 0 and sol.t == 0
    for _ in range(3):
        c.call()
    assert c.stats.failures == 1 and sol.t == 4 * K and net.calls == 0


def _fake_compare(errors):
    """A stand-in for compare_to_solver: errors[(case, tol_disp)] = (phi_l2,
    interface); records every (case, tol_disp) it is asked for."""
    asked = []

    def compare(sur, prm, f, calls, tol=None, tol_disp=None, repeats=1):
        asked.append((prm, tol_disp))
        l2, itf = errors[(prm, tol_disp)]
        return {"phi_l2": l2, "interface_max": itf, "speedup": 1.0 + tol_disp,
                "stats": {"calls": calls, "net_calls": calls // 2, "failures": 0}}
    return compare, asked


def test_calibration_takes_the_largest_tolerance_within_the_margin(monkeypatch):
    """Candidates are tried from the largest down and the first at which
    every case ends within margin x both bars is kept; a case inside the bars
    but outside the margin disqualifies a candidate, on either measure."""
    bar_l2, bar_if = surrogate.BAR_PHI_L2, surrogate.BAR_INTERFACE
    cands = (0.3, 0.1, 0.03)
    errors = {
        ("a", 0.3): (0.5 * bar_l2, 0.9 * bar_if), ("b", 0.3): (0.1 * bar_l2, 0.1 * bar_if),  # a: inside bar, not margin
        ("a", 0.1): (0.1 * bar_l2, 0.5 * bar_if), ("b", 0.1): (0.85 * bar_l2, 0.1 * bar_if),  # b: phi L2 past margin
        ("a", 0.03): (0.1 * bar_l2, 0.3 * bar_if), ("b", 0.03): (0.2 * bar_l2, 0.2 * bar_if),
    }
    compare, asked = _fake_compare(errors)
    monkeypatch.setattr(surrogate, "compare_to_solver", compare)
    res = surrogate.calibrate_tolerance(None, [("a", None), ("b", None)], calls=8, candidates=cands, margin=0.8)
    assert res["tol_disp"] == 0.03
    assert [r["tol_disp"] for r in res["candidates"]] == [0.3, 0.1, 0.03]
    assert [r["qualifies"] for r in res["candidates"]] == [False, False, True]
    assert res["candidates"][0]["interface_max_cells"] == 0.9 * bar_if
    assert res["candidates"][1]["phi_l2_max"] == 0.85 * bar_l2
    assert res["candidates"][2]["network_share"] == 0.5
    assert len(asked) == 6
    # once a candidate qualifies, the smaller ones are not run
    errors[("b", 0.1)] = (0.1 * bar_l2, 0.1 * bar_if)
    compare, asked = _fake_compare(errors)
    monkeypatch.setattr(surrogate, "compare_to_solver", compare)
    res = surrogate.calibrate_tolerance(None, [("a", None), ("b", None)], calls=8, candidates=cands, margin=0.8)
    assert res["tol_disp"] == 0.1 and len(res["candidates"]) == 2 and len(asked) == 4


def test_calibration_reports_none_when_no_candidate_qualifies(monkeypatch):
    bar_l2, bar_if = surrogate.BAR_PHI_L2, surrogate.BAR_INTERFACE
    errors = {("a", td): (0.1 * bar_l2, 1.2 * bar_if) for td in (0.2, 0.02)}
    compare, _ = _fake_compare(errors)
    monkeypatch.setattr(surrogate, "compare_to_solver", compare)
    res = surrogate.calibrate_tolerance(None, [("a", None)], calls=8, candidates=(0.02, 0.2))
    assert res["tol_disp"] is None
    assert [r["tol_disp"] for r in res["candidates"]] == [0.2, 0.02]
    assert not any(r["qualifies"] for r in res["candidates"])
