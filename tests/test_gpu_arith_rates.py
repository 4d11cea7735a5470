"""combo_arith_rates: the FP64 and FP32 FMA throughput the arithmetic-bound
kernels are measured against.  Checks only what holds on any GPU of this
class: both rates positive and finite, FP32 well above FP64, and the FP32
rate below the nominal bound of 152 SMs x 128 FMA lanes x 2 FLOPs x 2.1 GHz
(with margin for another part)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_arith_rates_are_plausible():
    from paper_2204_13624_gb300 import build, combo

    build.build()
    combo.load()
    r64, r32 = combo.arith_rates()
    assert math.isfinite(r64) and math.isfinite(r32)
    assert r64 > 0.0 and r32 > 0.0
    assert r32 > 4.0 * r64
    assert r32 < 2.0 * 152 * 128 * 2 * 2.1e9 / 1e12
