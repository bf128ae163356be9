"""The device probes the roofline figures are measured against: the FMA
throughput in FP32 and FP64 (mmp_probe_fma) and the fine step's arithmetic
without the cross-CTA exchange (mmp_probe_step), run through the C-ABI.
They time work, so the checks are sanity bounds, not values."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rates(mmplib):
    t32 = mmplib.mmp_probe_fma("mixed")
    t64 = mmplib.mmp_probe_fma("fp64")
    assert math.isfinite(t32) and math.isfinite(t64)
    assert t32 > 0.0 and t64 > 0.0
    assert t32 > t64  # FP64 issues at a fraction of the FP32 rate on this chip


def test_step_probe_rates(mmplib):
    regs = mmplib.mmp_probe_step(0)
    smem = mmplib.mmp_probe_step(1)
    assert math.isfinite(regs) and math.isfinite(smem)
    assert regs > 0.0 and smem > 0.0
    # the shared-memory form adds a load, a store and a barrier per step; it
    # cannot be much faster than the same arithmetic in registers
    assert smem < 1.25 * regs, (regs, smem)
