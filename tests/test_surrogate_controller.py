"""The surrogate controller's decisions, on the CPU with stand-ins for the
network and the solver.

The controller (a check every ``check_every`` calls against K solver steps
from the same start, roll-back to the last verified state and recomputation
by the solver when the check fails, then ``cooldown`` windows on the solver
alone) is host logic.  Here the state is two numbers, the time t in steps and
a "drift" that only the network adds; the solver advances t exactly and adds
nothing.  So after every call t must equal calls * K, and the drift tells
which network results were kept.
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
