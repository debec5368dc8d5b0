"""The measured rates that bound kernels of the library.

gpe2p_fma_rate (the FP64 path's bound): both precisions are positive and
finite, FP32 is the faster, and the FP32 rate lies below the nominal peak of
the part (152 SMs x 128 FP32 lanes x 2 operations x 2.07 GHz = 80.5
TFLOP/s), so the chains are not optimised away.

gpe2p_mma_rate (the surrogate convolutions' bound): the tensor cores of an
SM do at most 4096 dense BF16 multiply-adds per cycle (152 SMs at about
1.8 GHz give the nominal 2.25 PFLOP/s), so an MMA of 128 x N x 16 takes at
least 128 N 16 / 4096 cycles; and a second issuing thread never makes the
SM slower."""
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


def test_mma_issue_rates():
    build.build()
    rows = {}
    for n in (32, 64, 128, 256):
        for k in (1, 2, 4):
            if n * k > 512:
                continue
            c = gpe2p.mma_rate(n, k)
            rows[n, k] = c
            print(f"N {n:3d} issuers {k}: {c:6.1f} cycles per MMA per SM, {128 * n * 16 / c:6.0f} MAC/cycle")
            assert math.isfinite(c) and c >= 128 * n * 16 / 4096 * 0.98
    for n in (32, 64, 128):
        assert rows[n, 2] <= rows[n, 1] * 1.05
    with pytest.raises(gpe2p.GPE2PError):
        gpe2p.mma_rate(48, 1)
    with pytest.raises(gpe2p.GPE2PError):
        gpe2p.mma_rate(256, 4)
