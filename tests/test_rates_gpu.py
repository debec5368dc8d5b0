"""The measured multiply-add rates (gpe2p_fma_rate) that bound the FP64 path:
both are positive and finite, FP32 is the faster, and the FP32 rate lies
below the nominal peak of the part (152 SMs x 128 FP32 lanes x 2 operations
x 2.07 GHz = 80.5 TFLOP/s), so the chains are not optimised away."""
from __future__ import annotations

import math

import pytest

from paper_2011_00814_gb300 import build, gpe2p

pytestmark = pytest.mark.gpu


def test_fma_rates():
    build.build()
    r64 = gpe2p.fma_rate(64)["flops_per_s"]
    r32 = gpe2p.fma_rate(32)["flops_per_s"]
    print(f"FP64 {r64 / 1e12:.3f} TFLOP/s, FP32 {r32 / 1e12:.2f} TFLOP/s")
    assert math.isfinite(r64) and math.isfinite(r32)
    assert 0.0 < r64 < r32
    assert r32 < 1.02 * 152 * 128 * 2 * 2.07e9
    with pytest.raises(gpe2p.GPE2PError):
        gpe2p.fma_rate(16)
