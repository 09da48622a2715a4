"""The FP64 rate measurement used as the FP64 step's roofline denominator:
positive, finite and of the order of a GB300's dense FP64 rate (nominal
1.25 TFLOP/s), and steady from call to call."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_measure_fp64_rate():
    from paper_1902_02999_gb300 import measure_fp64
    a, b = measure_fp64(), measure_fp64()
    print("FP64 FMA rate: %.3f, %.3f TFLOP/s" % (a, b))
    assert math.isfinite(a) and 0.2 < a < 10.0
    assert abs(a - b) <= 0.1 * a
