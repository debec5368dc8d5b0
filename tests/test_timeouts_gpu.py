"""The bounded waits of the 3D kernels and of the tcgen05 convolutions, made
to report a timeout from the host (GPE2P_FAULT_LOSE_COPY).

3D kernels: in every block of the chosen kernel the first wait of the chosen
kind completes and is then treated as timed out, as if its copy had been
lost.  The block records the error, waits for its other copies in flight and
returns; the next diagnostics report GPE2P_ETIMEOUT.  After GPE2P_FAULT_CLEAR
and gpe2p_init_fields the same handle steps cleanly again, bit for bit as a
handle that never saw the switch.

Convolutions: the same for the first wait of every CTA for a filled pipeline
stage (gpe2p_net_fault).

Nothing faults on the GPU: only the kernels' own timeout bookkeeping runs."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2011_00814_gb300 import build, gpe2p, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    gpe2p.lib()


def _case(ch_advection=0):
    prm, f = inputs.bubble3d(40, 24, 36, R=6.0, gap=6.0)
    return dict(prm, precision=32, ch_advection=ch_advection), f


def _clean(prm, f, n):
    with gpe2p.Solver(prm) as s:
        s.set_phi_accumulation(gpe2p.PHI_ACC_FP32)
        s.init_fields(f)
        s.advance(n)
        return s.read_fields()


@pytest.mark.parametrize("bit,adv", [(gpe2p.LOSE_FLOW_RING, 0), (gpe2p.LOSE_CH_RING, 0), (gpe2p.LOSE_MU_RING, 0),
                                     (gpe2p.LOSE_CH_POINTS, 0), (gpe2p.LOSE_CH_RING, 1)])
def test_lost_copy_reports_timeout_and_the_handle_recovers(bit, adv):
    prm, f = _case(adv)
    want = _clean(prm, f, 3)
    with gpe2p.Solver(prm) as s:
        # one fixed accumulation policy on both handles: the automatic one
        # could switch at a different diagnostics call on each
        s.set_phi_accumulation(gpe2p.PHI_ACC_FP32)
        s.init_fields(f)
        s.step()
        assert s.diagnostics()["nan_flag"] == 0
        s.fault(gpe2p.FAULT_LOSE_COPY, bit)
        s.step()
        with pytest.raises(gpe2p.GPE2PError) as e:
            s.diagnostics()
        assert e.value.code == gpe2p.ETIMEOUT
        s.fault(gpe2p.FAULT_CLEAR)
        s.init_fields(f)
        s.advance(3)
        got = s.read_fields()
    for k in ("phi", "p", "u", "v", "w", "mu"):
        assert np.array_equal(got[k], want[k]), k


def test_lose_copy_is_refused_where_it_does_not_apply():
    prm = dict(inputs.base_params(2, 16, 16), precision=32)
    with gpe2p.Solver(prm) as s:
        with pytest.raises(gpe2p.GPE2PError) as e:
            s.fault(gpe2p.FAULT_LOSE_COPY, 1)
        assert e.value.code == gpe2p.EINVAL
    prm3, _ = _case()
    with gpe2p.Solver(prm3) as s:
        with pytest.raises(gpe2p.GPE2PError):
            s.fault(gpe2p.FAULT_LOSE_COPY, 16)
        with pytest.raises(gpe2p.GPE2PError):
            s.fault(gpe2p.FAULT_SKIP_BARRIER, 0)


@pytest.mark.parametrize("shape", [(3, [16, 32, 64], 32, 32, 2), (4, [32, 64, 128, 256], 64, 64, 2)])
def test_lost_stage_of_the_tcgen05_convolutions_reports_timeout_and_the_net_recovers(shape):
    """The tcgen05 convolutions' pipeline waits (gpe2p_net_fault): with the
    switch on, the first wait of every CTA for a filled stage reports a
    timeout; the other roles give up their waits and the CTA returns, and the
    forward's gpe2p_net_sync and gpe2p_net_gradients report GPE2P_ETIMEOUT.
    After GPE2P_FAULT_CLEAR the same handle computes the forward bit for bit
    as before the switch.  On the small net the layers keep their weights in
    shared memory; on the 4-level net some stream them through the ring."""
    import torch
    L, ch, h, w, b = shape
    rng = np.random.default_rng(4)
    with gpe2p.Net(L, ch, 4, 4, h, w, b, seed=3) as net:
        net.set_backend(True)
        x = torch.from_numpy(rng.normal(size=(b, h, w, 4)).astype(np.float32)).cuda()
        t = torch.from_numpy(rng.normal(size=(b, h, w, 4)).astype(np.float32)).cuda()
        y0 = torch.empty((b, h, w, 4), dtype=torch.float32, device="cuda")
        net.forward(x, y0, b)
        net.sync()
        net.fault(gpe2p.FAULT_LOSE_COPY, 1)
        y1 = torch.empty_like(y0)
        net.forward(x, y1, b)
        with pytest.raises(gpe2p.GPE2PError) as e:
            net.sync()
        assert e.value.code == gpe2p.ETIMEOUT
        with pytest.raises(gpe2p.GPE2PError) as e:
            net.gradients(x, t, b)
        assert e.value.code == gpe2p.ETIMEOUT
        net.fault(gpe2p.FAULT_CLEAR)
        y2 = torch.empty_like(y0)
        net.forward(x, y2, b)
        net.sync()
        assert torch.equal(y2, y0)
        with pytest.raises(gpe2p.GPE2PError) as e:
            net.fault(gpe2p.FAULT_SKIP_BARRIER, 0)
        assert e.value.code == gpe2p.EINVAL
